// Broken-line helix fit of every selected ntuplet, written straight into the compact output.
//
// Steps (V. Blobel, NIM A 566 (2006) 14, as read for this library):
//  1. local frame at hit 0; reference circle through hits 0, n/2, n-1 (centre C, radius R0,
//     orientation sgn = sign D, charge -sgn);
//  2. path lengths s_i (angle about C times R0) and outward residuals
//     y_i = (|p_i|^2 - 2 p_i.C) / (|p_i - C| + R0)  (cancellation-free |p_i - C| - R0);
//  3. Highland scattering angle from the reference momentum, kink variances projected by
//     1 + cot^2 (transverse) and (1 + cot^2)^2 (line);
//  4. transverse broken line (offsets u_i + curvature correction delta) and line broken line
//     (z_i), each the minimiser of its chi2, solved in the parameters (kinks, x_0, slope
//     [, delta]): the kink block (kink weights on its diagonal) by Cholesky, bordered by the
//     global unknowns, which its Schur complement gives;
//  5. fitted circle at hit 0 and its point of closest approach to the z axis.
// Precision modes: FP64 (all steps double), MIXED (arithmetic double, transcendentals float),
// FP32 (all float), SPLIT (steps 1-3 in float, on a chord frame whose differences are
// error-free; the normal matrices and their Cholesky factorisation in double-float arithmetic
// when every hit is on a barrel layer, in double otherwise; the conversion in double; tracks
// where the float reference circle would limit the accuracy are refitted in FP64).  The hit
// count is a template parameter, so every array lives in registers.
#include "pxr_dev.cuh"

namespace pxr {

constexpr double kKpt = 0.299792458e-2;   // pT [GeV] = K B [T] R [cm]

template <typename T>
__device__ __forceinline__ T sqrt_t(T v) { return sqrt(v); }
template <>
__device__ __forceinline__ float sqrt_t<float>(float v) { return sqrtf(v); }
template <typename T>
__device__ __forceinline__ T rsqrt_t(T v) { return rsqrt(v); }
template <>
__device__ __forceinline__ float rsqrt_t<float>(float v) { return rsqrtf(v); }

// Transcendentals in float (FT = true) or in the argument's own type.
template <bool FT, typename T>
__device__ __forceinline__ T atan2_t(T y, T x)
{
    if constexpr (FT) return T(atan2f(float(y), float(x)));
    else return atan2(y, x);
}
template <bool FT, typename T>
__device__ __forceinline__ T log_t(T v) { return FT ? T(logf(float(v))) : log(v); }

// Turning angle about the reference centre, for the arc lengths.  A float arctangent is good to
// ~1e-7 relative, and a nearly straight fitted track (whose curvature is a small difference of
// inverse radii) amplifies that in pT; so with float transcendentals the small angles, where
// that happens (|angle| < 0.25 rad), come from the arctangent series in the working precision
// (terms to t^17: truncation below 4e-13 relative), the larger ones from the float function.
template <bool FT, typename T>
__device__ __forceinline__ T arc_angle(T y, T x)
{
    if (FT && x > T(0) && fabs(y) < T(0.25) * x) {
        const T t = y / x, t2 = t * t;
        T p = T(1.0 / 17.0);
        p = p * t2 - T(1.0 / 15.0);
        p = p * t2 + T(1.0 / 13.0);
        p = p * t2 - T(1.0 / 11.0);
        p = p * t2 + T(1.0 / 9.0);
        p = p * t2 - T(1.0 / 7.0);
        p = p * t2 + T(1.0 / 5.0);
        p = p * t2 - T(1.0 / 3.0);
        p = p * t2 + T(1.0);
        return t * p;
    }
    return atan2_t<FT>(y, x);
}

struct FitOut {
    double pt, phi, cot, dxy, dz, chi2;
    int8_t q, status;
};

// In-place Cholesky factor L L^T of a small symmetric positive definite matrix (lower triangle
// used); the diagonal receives the reciprocals of L's diagonal (the solves multiply).
template <int K, typename T>
__device__ __forceinline__ bool chol_factor(T (&A)[K][K])
{
#pragma unroll
    for (int j = 0; j < K; ++j) {
        T d = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
        if (!(d > T(0))) return false;
        const T il = rsqrt_t(d);
        A[j][j] = il;
#pragma unroll
        for (int i = j + 1; i < K; ++i) {
            T t = A[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= A[i][k] * A[j][k];
            A[i][j] = t * il;
        }
    }
    return true;
}

// y = L^-1 b and x = L^-T y with the factor of chol_factor.
template <int K, typename T>
__device__ __forceinline__ void chol_lower(const T (&L)[K][K], T (&b)[K])
{
#pragma unroll
    for (int i = 0; i < K; ++i) {
        T t = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t -= L[i][k] * b[k];
        b[i] = t * L[i][i];
    }
}
template <int K, typename T>
__device__ __forceinline__ void chol_upper(const T (&L)[K][K], T (&y)[K])
{
#pragma unroll
    for (int i = K - 1; i >= 0; --i) {
        T t = y[i];
#pragma unroll
        for (int k = i + 1; k < K; ++k) t -= L[k][i] * y[k];
        y[i] = t * L[i][i];
    }
}

// Broken line over N points (arc-length steps h[i] = s[i+1] - s[i]): measurements meas with
// weights w, a kink at each inner point j with weight wk[j] (reciprocal variance), and (CURV) one
// curvature correction delta.  Kink j = (x_{j+1} - x_j)/h_j - (x_j - x_{j-1})/h_{j-1}
// + CURV (h_{j-1} + h_j)/2 delta; the fit minimises sum w (meas - x)^2 + sum wk kink^2.
// It is solved in the parameters theta = (kinks, x_0, first slope, [delta]), which give the
// paths one to one: x_i = x_0 + slope (s_i - s_0) + sum_{0<j<i} (kink_j - CURV c_j delta)
// (s_i - s_j), c_j = (h_{j-1} + h_j)/2.  The normal matrix keeps the kink weights (up to ~1e20
// for nearly straight tracks) on the diagonal of its kink block, apart from the measurement
// weights (~1e6) that fill the rest: the kink block is factored (Cholesky), the border of the
// global unknowns (x_0, slope[, delta]) eliminated through its Schur complement, factored in turn.
// Returns the offsets x, the curvature correction and the chi2 at the minimum; with CV, also the
// covariance of (x_0, x_1[, delta]) (the Schur complement's inverse carried to x_1 = x_0 + h_0
// slope: cv = c00, c01, c11 and, with CURV, c0d, c1d, cdd).
template <int N, bool CURV, typename T, bool CV = false>
__device__ __forceinline__ bool broken_line_n(const T (&h)[N], const T (&meas)[N],
                                              const T (&w)[N], const T (&wk)[N], T (&x)[N],
                                              T &delta, T &chi2, T *cv = nullptr)
{
    constexpr int K = N - 2;                 // kinks
    constexpr int G = CURV ? 3 : 2;          // x_0, slope, [delta]
    T S[N], jd[N];                           // s_i - s_0; d x_i / d delta
    S[0] = T(0);
#pragma unroll
    for (int i = 1; i < N; ++i) S[i] = S[i - 1] + h[i - 1];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T a = T(0);
#pragma unroll
        for (int j = 1; j < i && j + 1 < N; ++j) a -= T(0.5) * (h[j - 1] + h[j]) * (S[i] - S[j]);
        jd[i] = a;
    }
    // d x_i / d theta: kink j -> (S_i - S_j)_+, x_0 -> 1, slope -> S_i, delta -> jd_i
    auto jk = [&](int i, int j) { return i > j ? S[i] - S[j] : T(0); };   // j = 1..K
    auto jg = [&](int i, int c) { return c == 0 ? T(1) : c == 1 ? S[i] : jd[i]; };
    T A[K][K], B[K][G], Gm[G][G], rb[K], rg[G];
#pragma unroll
    for (int a = 0; a < K; ++a) {
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            T v = a == b ? wk[a + 1] : T(0);
#pragma unroll
            for (int i = 0; i < N; ++i) v += w[i] * jk(i, a + 1) * jk(i, b + 1);
            A[a][b] = v;
        }
#pragma unroll
        for (int c = 0; c < G; ++c) {
            T v = T(0);
#pragma unroll
            for (int i = 0; i < N; ++i) v += w[i] * jk(i, a + 1) * jg(i, c);
            B[a][c] = v;
        }
        T v = T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) v += w[i] * jk(i, a + 1) * meas[i];
        rb[a] = v;
    }
#pragma unroll
    for (int c = 0; c < G; ++c) {
#pragma unroll
        for (int d = 0; d <= c; ++d) {
            T v = T(0);
#pragma unroll
            for (int i = 0; i < N; ++i) v += w[i] * jg(i, c) * jg(i, d);
            Gm[c][d] = v;
        }
        T v = T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) v += w[i] * jg(i, c) * meas[i];
        rg[c] = v;
    }
    // kink block: A = L L^T; Y = L^-1 B, y = L^-1 rb; Schur complement Gm - Y^T Y
    if (!chol_factor<K, T>(A)) return false;
    chol_lower<K, T>(A, rb);
#pragma unroll
    for (int c = 0; c < G; ++c) {
        T col[K];
#pragma unroll
        for (int a = 0; a < K; ++a) col[a] = B[a][c];
        chol_lower<K, T>(A, col);
#pragma unroll
        for (int a = 0; a < K; ++a) B[a][c] = col[a];
    }
#pragma unroll
    for (int c = 0; c < G; ++c) {
#pragma unroll
        for (int d = 0; d <= c; ++d) {
            T v = Gm[c][d];
#pragma unroll
            for (int a = 0; a < K; ++a) v -= B[a][c] * B[a][d];
            Gm[c][d] = v;
        }
        T v = rg[c];
#pragma unroll
        for (int a = 0; a < K; ++a) v -= B[a][c] * rb[a];
        rg[c] = v;
    }
    if (!chol_factor<G, T>(Gm)) return false;
    T tg[G];
#pragma unroll
    for (int c = 0; c < G; ++c) tg[c] = rg[c];
    chol_lower<G, T>(Gm, tg);
    chol_upper<G, T>(Gm, tg);
    // kinks: L^T beta = y - Y theta_g
#pragma unroll
    for (int a = 0; a < K; ++a) {
        T v = rb[a];
#pragma unroll
        for (int c = 0; c < G; ++c) v -= B[a][c] * tg[c];
        rb[a] = v;
    }
    chol_upper<K, T>(A, rb);
    delta = CURV ? tg[G - 1] : T(0);
    T c2 = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T v = tg[0] + S[i] * tg[1];
        if (CURV) v += jd[i] * tg[G - 1];
#pragma unroll
        for (int a = 0; a < K; ++a) v += jk(i, a + 1) * rb[a];
        x[i] = v;
        const T r = meas[i] - v;
        c2 += w[i] * r * r;
    }
#pragma unroll
    for (int a = 0; a < K; ++a) c2 += wk[a + 1] * rb[a] * rb[a];
    chi2 = c2;
    if constexpr (CV) {
        // the globals' covariance: the inverse of the Schur complement, columns by solves
        T Ci[G][G];
#pragma unroll
        for (int c = 0; c < G; ++c) {
            T e[G];
#pragma unroll
            for (int d = 0; d < G; ++d) e[d] = c == d ? T(1) : T(0);
            chol_lower<G, T>(Gm, e);
            chol_upper<G, T>(Gm, e);
#pragma unroll
            for (int d = 0; d < G; ++d) Ci[d][c] = e[d];
        }
        const T h0 = h[0];
        cv[0] = Ci[0][0];
        cv[1] = Ci[0][0] + h0 * Ci[0][1];
        cv[2] = Ci[0][0] + T(2) * h0 * Ci[0][1] + h0 * h0 * Ci[1][1];
        if (CURV) {
            cv[3] = Ci[0][G - 1];
            cv[4] = Ci[0][G - 1] + h0 * Ci[1][G - 1];
            cv[5] = Ci[G - 1][G - 1];
        }
    }
    return true;
}

// Elimination of one view's normal equations in the kink parametrisation, the steps of
// broken_line_n: the kink block A (K x K, lower part) factored, the border B (K x G) and the
// right-hand side rb carried through it, the globals' Schur complement Gm - Y^T Y (G x G) factored
// and solved, then the kinks.  On return tg holds the globals and rb the kinks.
template <int K, int G, typename T>
__device__ __forceinline__ bool bl_eliminate(T (&A)[K][K], T (&B)[K][G], T (&Gm)[G][G],
                                             T (&rb)[K], T (&rg)[G], T (&tg)[G])
{
    if (!chol_factor<K, T>(A)) return false;
    chol_lower<K, T>(A, rb);
#pragma unroll
    for (int c = 0; c < G; ++c) {
        T col[K];
#pragma unroll
        for (int a = 0; a < K; ++a) col[a] = B[a][c];
        chol_lower<K, T>(A, col);
#pragma unroll
        for (int a = 0; a < K; ++a) B[a][c] = col[a];
    }
#pragma unroll
    for (int c = 0; c < G; ++c) {
#pragma unroll
        for (int d = 0; d <= c; ++d) {
            T v = Gm[c][d];
#pragma unroll
            for (int a = 0; a < K; ++a) v -= B[a][c] * B[a][d];
            Gm[c][d] = v;
        }
        T v = rg[c];
#pragma unroll
        for (int a = 0; a < K; ++a) v -= B[a][c] * rb[a];
        rg[c] = v;
    }
    if (!chol_factor<G, T>(Gm)) return false;
#pragma unroll
    for (int c = 0; c < G; ++c) tg[c] = rg[c];
    chol_lower<G, T>(Gm, tg);
    chol_upper<G, T>(Gm, tg);
#pragma unroll
    for (int a = 0; a < K; ++a) {
        T v = rb[a];
#pragma unroll
        for (int c = 0; c < G; ++c) v -= B[a][c] * tg[c];
        rb[a] = v;
    }
    chol_upper<K, T>(A, rb);
    return true;
}

// Add t to the running sum v, or start the sum with it (the unrolled loops below decide at
// compile time which terms exist, so no sum starts from a literal zero).
template <typename T>
__device__ __forceinline__ void acc(T &v, bool &started, const T &t)
{
    if (started) {
        v += t;
    } else {
        v = t;
        started = true;
    }
}

// Both views of a track whose hits share one measurement weight per view (wT, wL) and one kink
// weight per view (every hit on a barrel layer): the minimisers of broken_line_n for the two
// views.  Divided by its measurement weight, a view's normal matrix is J^T J with
// lam = kink weight / measurement weight added on the kink diagonal, where J (d x_i / d theta) is
// the same arc-length geometry in both views; the transverse view has the extra curvature
// column.  J^T J is therefore built once, with no weights in it, and each view adds its lam and
// right-hand side.  Returns both views' fitted points, delta, and the summed chi2 of both views
// (the measurement weights put back).
template <int N, typename T>
__device__ __forceinline__ bool broken_line_pair(const T (&h)[N], const T (&mT)[N],
                                                 const T (&mL)[N], T wT, T wL, T lamT, T lamL,
                                                 T (&xT)[N], T (&xL)[N], T &delta, T &chi2)
{
    constexpr int K = N - 2;                 // kinks
    // J's structural zeros and ones are left out of every product and sum: d x_i / d kink j is
    // zero up to hit j + 1, d x_i / d slope (S_i = s_i - s_0) is zero at hit 0, d x_i / d delta
    // (jd_i) at hits 0 and 1, d x_i / d x_0 is one.  (A product with a literal zero cannot be
    // folded away in IEEE arithmetic; the results are the same bit for bit.)
    T S[N], jd[N];                           // s_i - s_0; d x_i / d delta
    S[0] = T(0);
    S[1] = h[0];
#pragma unroll
    for (int i = 2; i < N; ++i) S[i] = S[i - 1] + h[i - 1];
    jd[0] = jd[1] = T(0);
#pragma unroll
    for (int i = 2; i < N; ++i) {
        T a = -(T(0.5) * (h[0] + h[1]) * (S[i] - S[1]));
#pragma unroll
        for (int j = 2; j < i && j + 1 < N; ++j) a -= T(0.5) * (h[j - 1] + h[j]) * (S[i] - S[j]);
        jd[i] = a;
    }
    // D[a][i] = d x_i / d kink (a + 1) for i > a + 1
    T D[K][N];
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
        for (int i = a + 2; i < N; ++i) D[a][i] = S[i] - S[a + 1];
    auto gnz = [](int i, int c) { return c == 0 || i >= c; };             // (x_0, slope, delta)
    auto gv = [&](int i, int c) { return c == 1 ? S[i] : jd[i]; };        // (c > 0)
    // the shared geometry J^T J: kink block, border, globals (x_0, slope, delta)
    T A[K][K], B[K][3], Gm[3][3], rbT[K], rbL[K], rgT[3], rgL[2];
#pragma unroll
    for (int a = 0; a < K; ++a) {
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            T v;
            bool st = false;
#pragma unroll
            for (int i = a + 2; i < N; ++i) acc(v, st, D[a][i] * D[b][i]);
            A[a][b] = v;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T v;
            bool st = false;
#pragma unroll
            for (int i = a + 2; i < N; ++i)
                if (gnz(i, c)) acc(v, st, c == 0 ? D[a][i] : D[a][i] * gv(i, c));
            B[a][c] = v;
        }
        T vT, vL;
        bool st = false, sl = false;
#pragma unroll
        for (int i = a + 2; i < N; ++i) {
            acc(vT, st, D[a][i] * mT[i]);
            acc(vL, sl, D[a][i] * mL[i]);
        }
        rbT[a] = vT;
        rbL[a] = vL;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int d = 0; d <= c; ++d) {
            T v;
            bool st = false;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                if (!gnz(i, c) || !gnz(i, d)) continue;
                if (c == 0) acc(v, st, T(1));
                else if (d == 0) acc(v, st, gv(i, c));
                else acc(v, st, gv(i, c) * gv(i, d));
            }
            Gm[c][d] = v;
        }
        T vT, vL;
        bool st = false, sl = false;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (!gnz(i, c)) continue;
            acc(vT, st, c == 0 ? mT[i] : gv(i, c) * mT[i]);
            if (c < 2) acc(vL, sl, c == 0 ? mL[i] : gv(i, c) * mL[i]);
        }
        rgT[c] = vT;
        if (c < 2) rgL[c] = vL;
    }
    // each view: its kink weight ratio on the diagonal, then the elimination
    T AT[K][K], AL[K][K], BT[K][3], BL[K][2], GT[3][3], GL[2][2], tgT[3], tgL[2];
#pragma unroll
    for (int a = 0; a < K; ++a) {
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            AT[a][b] = a == b ? A[a][b] + lamT : A[a][b];
            AL[a][b] = a == b ? A[a][b] + lamL : A[a][b];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            BT[a][c] = B[a][c];
            if (c < 2) BL[a][c] = B[a][c];
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d <= c; ++d) {
            GT[c][d] = Gm[c][d];
            if (c < 2) GL[c][d] = Gm[c][d];
        }
    if (!bl_eliminate<K, 3, T>(AT, BT, GT, rbT, rgT, tgT)) return false;
    if (!bl_eliminate<K, 2, T>(AL, BL, GL, rbL, rgL, tgL)) return false;
    delta = tgT[2];
    T c2T = T(0), c2L = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T vT = tgT[0], vL = tgL[0];
        if (i >= 1) {
            vT += S[i] * tgT[1];
            vL += S[i] * tgL[1];
        }
        if (i >= 2) vT += jd[i] * tgT[2];
#pragma unroll
        for (int a = 0; a < K; ++a) {
            if (i < a + 2) continue;
            vT += D[a][i] * rbT[a];
            vL += D[a][i] * rbL[a];
        }
        xT[i] = vT;
        xL[i] = vL;
        const T rT = mT[i] - vT, rL = mL[i] - vL;
        c2T += rT * rT;
        c2L += rL * rL;
    }
    T kT = T(0), kL = T(0);
#pragma unroll
    for (int a = 0; a < K; ++a) {
        kT += rbT[a] * rbT[a];
        kL += rbL[a] * rbL[a];
    }
    chi2 = wT * (c2T + lamT * kT) + wL * (c2L + lamL * kL);
    return true;
}

// Geometry of the conversion: the reference circle (reciprocal radius, centre, orientation) in
// the frame of hit 0, the first arc-length step (and its reciprocal), hit 0, and K B.
template <typename T>
struct ConvGeom {
    T iR0, Cx, Cy, sgs, g0, ds0, X0, Y0, kB;
};

// Forward-mode derivatives: a value and its derivatives with respect to the five fitted values
// (u_0, u_1, delta, v_0, v_1).  The conversion below runs on it to give the exact Jacobian of
// the track parameters (the chain rule of each operation, no difference quotients).
struct D5 {
    double v, d[5];
    __device__ D5(double x = 0.0) : v(x) { for (int i = 0; i < 5; ++i) d[i] = 0.0; }
    __device__ explicit operator double() const { return v; }
};
__device__ __forceinline__ D5 operator+(const D5 &a, const D5 &b)
{ D5 r(a.v + b.v); for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
__device__ __forceinline__ D5 operator-(const D5 &a, const D5 &b)
{ D5 r(a.v - b.v); for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
__device__ __forceinline__ D5 operator-(const D5 &a)
{ D5 r(-a.v); for (int i = 0; i < 5; ++i) r.d[i] = -a.d[i]; return r; }
__device__ __forceinline__ D5 operator*(const D5 &a, const D5 &b)
{ D5 r(a.v * b.v); for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
__device__ __forceinline__ D5 operator/(const D5 &a, const D5 &b)
{ D5 r(a.v / b.v); for (int i = 0; i < 5; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v; return r; }
__device__ __forceinline__ bool operator>(const D5 &a, const D5 &b) { return a.v > b.v; }
__device__ __forceinline__ bool operator==(const D5 &a, const D5 &b) { return a.v == b.v; }
__device__ __forceinline__ bool isfinite(const D5 &a) { return ::isfinite(a.v); }
__device__ __forceinline__ D5 fabs(const D5 &a) { return a.v < 0.0 ? -a : a; }
__device__ __forceinline__ D5 sin(const D5 &a)
{ D5 r(::sin(a.v)); const double c = ::cos(a.v); for (int i = 0; i < 5; ++i) r.d[i] = c * a.d[i]; return r; }
__device__ __forceinline__ D5 cos(const D5 &a)
{ D5 r(::cos(a.v)); const double s = -::sin(a.v); for (int i = 0; i < 5; ++i) r.d[i] = s * a.d[i]; return r; }
__device__ __forceinline__ D5 atan2(const D5 &y, const D5 &x)
{
    D5 r(::atan2(y.v, x.v));
    const double q = 1.0 / (x.v * x.v + y.v * y.v);
    for (int i = 0; i < 5; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) * q;
    return r;
}
template <>
__device__ __forceinline__ D5 rsqrt_t<D5>(D5 a)
{
    D5 r(::rsqrt(a.v));
    const double k = -0.5 * r.v * r.v * r.v;
    for (int i = 0; i < 5; ++i) r.d[i] = k * a.d[i];
    return r;
}
// the overloads above must not hide the plain floating-point functions inside this namespace
using ::atan2;
using ::cos;
using ::fabs;
using ::isfinite;
using ::sin;

// Conversion of the fitted offsets u_0, u_1, curvature correction delta and line values v_0, v_1
// to the point of closest approach: curvature, direction at hit 0 turned by the fitted slope,
// fitted centre, PCA; false when the fitted curvature vanishes.  T carries the fitted values (a
// floating type, or D5 for their Jacobian); TG the geometry.
template <bool FT, typename T, typename TG>
__device__ __forceinline__ bool convert_core(const ConvGeom<TG> &G, T u0, T u1, T delta, T v0,
                                             T v1, T &pt, T &phi, T &cot, T &dxy, T &dz,
                                             int &qf)
{
    const T kappa = T(G.iR0) + delta;
    if (kappa == T(0) || !isfinite(kappa)) return false;
    const T R = T(1) / fabs(kappa);
    const T sgs = T(G.sgs);
    const T sgf = kappa > T(0) ? sgs : -sgs;
    const T ds0 = T(G.ds0);
    const T alpha = (u1 - u0) * T(G.g0) + T(0.5) * delta * ds0;
    const T nx = -T(G.Cx) * T(G.iR0), ny = -T(G.Cy) * T(G.iR0);
    const T tx = -sgs * ny, ty = sgs * nx;
    T ca, sa;
    if constexpr (FT) {
        // cos of a small angle rounds to 1 in float; 1 - 2 sin^2(a/2) keeps its deviation
        const T sh = T(sinf(float(alpha * T(0.5))));
        ca = T(1) - T(2) * sh * sh;
        sa = T(sinf(float(alpha)));
    } else {
        ca = cos(alpha);
        sa = sin(alpha);
    }
    const T n2x = nx * ca - tx * sa, n2y = ny * ca - ty * sa;
    const T P0x = u0 * nx, P0y = u0 * ny;
    const T rk = kappa > T(0) ? R : -R;                  // 1 / kappa
    const T Fx = P0x - n2x * rk, Fy = P0y - n2y * rk;
    const T rx = (P0x - Fx) * fabs(kappa), ry = (P0y - Fy) * fabs(kappa);
    const T wx = -T(G.X0) - Fx, wy = -T(G.Y0) - Fy;
    const T d2 = wx * wx + wy * wy;
    const T idist = rsqrt_t(d2);
    const T dist = d2 * idist;
    const T ex = wx * idist, ey = wy * idist;
    const T tpx = -sgf * ey, tpy = sgf * ex;
    cot = (v1 - v0) * T(G.g0);
    const T psi = atan2_t<FT>(sgf * (ex * ry - ey * rx), ex * rx + ey * ry);
    qf = sgf > T(0) ? -1 : 1;
    pt = T(G.kB) * R;
    phi = atan2_t<FT>(tpy, tpx);
    dxy = T(double(qf)) * (dist - R);
    dz = v0 - cot * (R * psi);
    return true;
}

template <bool FT, typename T>
__device__ __forceinline__ bool bl_convert(const ConvGeom<T> &G, T u0, T u1, T delta, T v0, T v1,
                                           FitOut &o)
{
    T pt, phi, cot, dxy, dz;
    int qf;
    if (!convert_core<FT, T, T>(G, u0, u1, delta, v0, v1, pt, phi, cot, dxy, dz, qf)) return false;
    o.pt = double(pt);
    o.phi = double(phi);
    o.cot = double(cot);
    o.dxy = double(dxy);
    o.dz = double(dz);
    o.q = (int8_t)qf;
    return true;
}

template <typename T>
__device__ __forceinline__ void bl_covariance(const ConvGeom<T> &G, T u0, T u1, T delta, T v0,
                                              T v1, const T *cvT, const T *cvL, double *cov15);

// TC: prefit + residuals + arc lengths; T: everything else (scattering, solves, conversion);
// FT: float transcendentals (angles and logarithms need ~1e-7 relative, far inside the
// tolerances).  Divisions and square roots are shared where the method allows (one reciprocal
// per arc-length step, one scattering angle per surface type, reciprocal Cholesky pivots): they
// are the costly operations of the double-precision path.
template <int N, typename TC, typename T, bool FT, bool COV>
__device__ __noinline__ void fit_n(const float *X, const float *Y, const float *Z,
                                   const uint8_t *L, const DevParams &p, FitOut &o,
                                   double *cov15)
{
    o = FitOut{0, 0, 0, 0, 0, 0, 0, 0};
    TC px[N], py[N];
    const TC x0 = TC(X[0]), y0 = TC(Y[0]);
#pragma unroll
    for (int i = 0; i < N; ++i) { px[i] = TC(X[i]) - x0; py[i] = TC(Y[i]) - y0; }
    constexpr int ib = N / 2, ic = N - 1;
    const TC ux = px[ib], uy = py[ib], vx = px[ic], vy = py[ic];
    const TC D = TC(2) * (ux * vy - uy * vx);
    if (D == TC(0)) { o.status = 1; return; }
    const TC uu = ux * ux + uy * uy, vv = vx * vx + vy * vy;
    const TC iD = TC(1) / D;
    const TC Cx = (uu * vy - vv * uy) * iD, Cy = (vv * ux - uu * vx) * iD;
    const TC R0 = sqrt_t(Cx * Cx + Cy * Cy);
    const TC sgn = D > TC(0) ? TC(1) : TC(-1);

    T s[N], yr[N], z[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const TC dx = px[i] - Cx, dy = py[i] - Cy;
        const TC pw = (px[i] * px[i] + py[i] * py[i]) - TC(2) * (px[i] * Cx + py[i] * Cy);
        if constexpr (FT) {
            // the denominator (|p - C| + R0 ~ 2 R0) needs only float's relative accuracy: the
            // residual keeps its ~1e-7 relative error, far below the hit resolution
            const float den = sqrtf(float(dx * dx + dy * dy)) + float(R0);
            yr[i] = T(pw) * T(1.0f / den);
        } else {
            yr[i] = T(pw / (sqrt_t(dx * dx + dy * dy) + R0));
        }
        const TC cr = -Cx * dy + Cy * dx;
        const TC dt = -Cx * dx - Cy * dy;
        s[i] = T(R0 * arc_angle<FT>(sgn * cr, dt));
        z[i] = T(Z[i]);
    }
    T g[N], h[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        h[i] = i + 1 < N ? s[i + 1] - s[i] : T(1);
        g[i] = T(1) / h[i];
    }

    // multiple scattering: one Highland angle per surface type (barrel, disk).  (Float weights
    // were measured to move dz of nearly straight fits by up to ~1e-4 relative: kept in T.)
    using W = T;
    const W cot0 = W(z[ic] - z[0]) / W(s[ic] - s[0]);
    const W sec2 = W(1) + cot0 * cot0;
    const T isec2 = T(W(1) / sec2);
    const W sec = sqrt_t(sec2);
    const W pmom = W(kKpt * p.bfield) * W(R0) * sec;
    const W a0 = W(0.0136) / pmom;
    const T wrphi = T(1.0 / (p.sigma_rphi * p.sigma_rphi));
    const T wz = T(1.0 / (p.sigma_z * p.sigma_z));
    bool any_disk = false;
#pragma unroll
    for (int i = 0; i < N; ++i) any_disk |= p.is_disk[L[i]] != 0;
    // reciprocal squared scattering angle on a surface crossed with path factor `path`
    auto inv_th2 = [&](W path) {
        const W xx = W(p.x_over_x0) * path;
        const T th0 = T(a0 * sqrt_t(xx) * (W(1) + W(0.038) * log_t<FT>(xx)));
        return T(1) / (th0 * th0);
    };
    const T ib2 = inv_th2(sec);
    T id2 = ib2, wdisk = wz;
    if (any_disk) {
        const W icot = W(1) / fabs(cot0);
        id2 = inv_th2(sec * icot);
        const T iz = T(1.0 / p.sigma_z) * T(icot);   // disk: sigma_r = sigma_z |cot|
        wdisk = iz * iz;
    }
    T wkT[N], wkL[N], wT[N], wL[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const bool dk = p.is_disk[L[i]] != 0;
        wT[i] = wrphi;
        wL[i] = dk ? wdisk : wz;
        const T it2 = dk ? id2 : ib2;
        wkT[i] = it2 * isec2;            // kink variance th0^2 (1 + cot^2)
        wkL[i] = it2 * isec2 * isec2;    // kink variance th0^2 (1 + cot^2)^2
    }
    // a kink variance that is zero or not a number (a weight that is not finite) is bad input
#pragma unroll
    for (int j = 1; j + 1 < N; ++j)
        if (!isfinite(wkT[j]) || !isfinite(wkL[j])) { o.status = 4; return; }

    T xT[N], xL[N], delta, dummy, chi2T, chi2L;
    T cvT[6], cvL[3];
    if (!broken_line_n<N, true, T, COV>(h, yr, wT, wkT, xT, delta, chi2T, cvT) ||
        !broken_line_n<N, false, T, COV>(h, z, wL, wkL, xL, dummy, chi2L, cvL)) {
        o.status = 3;
        return;
    }

    // conversion to the point of closest approach
    const T R0s = T(R0);
    const T iR0 = T(1) / R0s;
    const ConvGeom<T> G{iR0, T(Cx), T(Cy), T(sgn), g[0], h[0], T(X[0]), T(Y[0]),
                        T(kKpt * p.bfield)};
    if (!bl_convert<FT, T>(G, xT[0], xT[1], delta, xL[0], xL[1], o)) { o.status = 2; return; }
    o.chi2 = double(chi2T + chi2L);
    o.status = 0;
    if constexpr (COV) bl_covariance<T>(G, xT[0], xT[1], delta, xL[0], xL[1], cvT, cvL, cov15);
}

// Covariance of (q/pT, phi, cot, dxy, dz): the fitted values' covariance (the blocks of the
// inverse normal matrices; the two broken lines are independent) through the conversion's
// Jacobian (forward-mode derivatives in FP64).  v0, v1: the line values the conversion took.
template <typename T>
__device__ __forceinline__ void bl_covariance(const ConvGeom<T> &G, T u0, T u1, T delta, T v0,
                                              T v1, const T *cvT, const T *cvL, double *cov15)
{
    {
        double C[5][5];
#pragma unroll
        for (int a = 0; a < 5; ++a)
#pragma unroll
            for (int c = 0; c < 5; ++c) C[a][c] = 0.0;
        C[0][0] = cvT[0]; C[0][1] = C[1][0] = cvT[1]; C[1][1] = cvT[2];
        C[0][2] = C[2][0] = cvT[3]; C[1][2] = C[2][1] = cvT[4]; C[2][2] = cvT[5];
        C[3][3] = cvL[0]; C[3][4] = C[4][3] = cvL[1]; C[4][4] = cvL[2];
        const ConvGeom<double> Gd{double(G.iR0), double(G.Cx), double(G.Cy), double(G.sgs),
                                  double(G.g0), double(G.ds0), double(G.X0), double(G.Y0),
                                  double(G.kB)};
        D5 q0[5];
        q0[0] = D5(double(u0));
        q0[1] = D5(double(u1));
        q0[2] = D5(double(delta));
        q0[3] = D5(double(v0));
        q0[4] = D5(double(v1));
#pragma unroll
        for (int k = 0; k < 5; ++k) q0[k].d[k] = 1.0;
        D5 pt, phi, cot, dxy, dz;
        int qf;
        const bool ok = convert_core<false, D5, double>(Gd, q0[0], q0[1], q0[2], q0[3], q0[4],
                                                        pt, phi, cot, dxy, dz, qf);
        const D5 qpt = D5(double(qf)) / pt;
        double J[5][5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            J[0][k] = qpt.d[k];
            J[1][k] = phi.d[k];
            J[2][k] = cot.d[k];
            J[3][k] = dxy.d[k];
            J[4][k] = dz.d[k];
        }
        int w = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = i; j < 5; ++j) {
                double acc = 0.0;
#pragma unroll
                for (int a = 0; a < 5; ++a)
#pragma unroll
                    for (int c = 0; c < 5; ++c) acc += J[i][a] * C[a][c] * J[j][c];
                cov15[w++] = ok ? acc : __longlong_as_double(0x7FF8000000000000LL);
            }
    }
}

template <typename TC, typename T, bool FT, bool COV>
__device__ __forceinline__ void fit_track(int n, const float *X, const float *Y, const float *Z,
                                          const uint8_t *L, const DevParams &p, FitOut &o,
                                          double *cov15)
{
    switch (n) {
    case 3: fit_n<3, TC, T, FT, COV>(X, Y, Z, L, p, o, cov15); break;
    case 4: fit_n<4, TC, T, FT, COV>(X, Y, Z, L, p, o, cov15); break;
    case 5: fit_n<5, TC, T, FT, COV>(X, Y, Z, L, p, o, cov15); break;
    case 6: fit_n<6, TC, T, FT, COV>(X, Y, Z, L, p, o, cov15); break;
    default: o = FitOut{0, 0, 0, 0, 0, 0, 0, 4};
    }
}

// ---- SPLIT: float bulk, double normal equations, factorisation and conversion ----
// Error-free transformations (Knuth's two-sum; the product's rounding error from a fused
// multiply-add): a + b = s + e and a b = p + e exactly.  The _rn intrinsics are never contracted
// or reassociated.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// ---- double-float arithmetic (a value as the unevaluated sum hi + lo of two floats) ----
// The error-free transformations of Knuth (sum) and Dekker (product, here with a fused
// multiply-add) give the rounding error of one float operation as another float; carrying it
// gives about 48 significant bits at float speed, where GB300's FP64 pipe runs at 1/64 of its
// FP32 rate.  Every operation is written with explicit round-to-nearest intrinsics, so that no
// step is contracted or reassociated.  Renormalised results (|lo| <= half an ulp of hi).
struct df64 {
    float hi, lo;
    __device__ df64() : hi(0.f), lo(0.f) {}
    __device__ df64(float h, float l) : hi(h), lo(l) {}
    __device__ df64(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df_fast(float s, float e)        // |s| >= |e|
{
    const float t = __fadd_rn(s, e);
    return df64(t, __fsub_rn(e, __fsub_rn(t, s)));
}
__device__ __forceinline__ df64 operator+(const df64 &a, const df64 &b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    float t, f;
    two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    const df64 u = df_fast(s, e);
    return df_fast(u.hi, __fadd_rn(u.lo, f));
}
__device__ __forceinline__ df64 operator-(const df64 &a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(const df64 &a, const df64 &b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(const df64 &a, const df64 &b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast(p, e);
}
__device__ __forceinline__ df64 &operator+=(df64 &a, const df64 &b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, const df64 &b) { return a = a - b; }
__device__ __forceinline__ bool operator>(const df64 &a, const df64 &b)
{
    return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
__device__ __forceinline__ bool isfinite(const df64 &a) { return ::isfinite(a.hi); }
// 1 / sqrt(a): the float estimate, then one Newton step y + y (1 - a y^2) / 2 in double-float
// (the estimate's ~23 bits doubled)
template <>
__device__ __forceinline__ df64 rsqrt_t<df64>(df64 a)
{
    const df64 y(rsqrtf(a.hi), 0.f);
    const df64 r = df64(1.0) - a * (y * y);
    return y + y * (r * df64(0.5f, 0.f));
}

// The refit of the tracks the float front end does not take: the same fit in FP64 (out of
// line; rare, so its cost does not matter, and a nearly straight fit from a bent reference
// amplifies any float rounding, transcendentals included).
template <int N, bool COV>
__device__ __forceinline__ void fit_refit64(const float *X, const float *Y, const float *Z,
                                            const uint8_t *L, const DevParams &p, FitOut &o,
                                            double *cov15)
{
    fit_n<N, double, double, false, COV>(X, Y, Z, L, p, o, cov15);
}

// Float front end on the chord frame of hits 0 and n-1: every hit's offset from hit 0 is
// carried exactly as two floats (two-sum), its components along the chord (a) and across it
// (b) follow, b with the products' rounding errors added back (so b, the small coordinate the
// curvature lives in, keeps float's relative accuracy however straight the track is).  The
// reference circle through hits 0, n/2, n-1, the outward residuals (the cancellation-free form
// (|q|^2 - 2 q.C) / (|q - C| + R0), exact for the circle of centre C through hit 0 whatever the
// rounding of C), the arc lengths, the weights and the Highland kinks are float; the two normal
// matrices are formed from these float values in double and factorised in double (the kink
// block, then the Schur complement of the global unknowns: a float normal matrix holds the
// measurement geometry of a nearly straight track too coarsely), and the conversion runs in
// double on the reference centre turned back to the global frame.  The fitted curvature inherits float's
// relative error of the reference curvature 1/R0 (a few 1e-7), so a track whose fitted
// curvature is more than ten times smaller than 1/R0 (a nearly straight fit from a bent
// reference) is refitted in FP64, as is any track the float front end cannot take (degenerate
// geometry, a failed factorisation).
template <int N, bool COV>
__device__ __noinline__ void fit_split_n(const float *X, const float *Y, const float *Z,
                                         const uint8_t *L, const DevParams &p, FitOut &o,
                                         double *cov15)
{
    constexpr int ib = N / 2, ic = N - 1;
    o = FitOut{0, 0, 0, 0, 0, 0, 0, 0};
    // 1. exact offsets from hit 0, the chord frame
    float dxh[N], dxl[N], dyh[N], dyl[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i == 0) { dxh[0] = dxl[0] = dyh[0] = dyl[0] = 0.f; continue; }
        two_sum(X[i], -X[0], dxh[i], dxl[i]);
        two_sum(Y[i], -Y[0], dyh[i], dyl[i]);
    }
    const float l2 = __fmaf_rn(dxh[ic], dxh[ic], __fmul_rn(dyh[ic], dyh[ic]));
    bool ok = l2 > 0.f && l2 < 1e30f;
    const float il = rsqrtf(l2);
    const float tx = dxh[ic] * il, ty = dyh[ic] * il;
    float a[N], b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i == 0) { a[0] = b[0] = 0.f; continue; }
        a[i] = __fmaf_rn(dxh[i], tx, __fmaf_rn(dyh[i], ty, __fmaf_rn(dxl[i], tx, dyl[i] * ty)));
        const float p1 = __fmul_rn(dxh[i], -ty), e1 = __fmaf_rn(dxh[i], -ty, -p1);
        const float p2 = __fmul_rn(dyh[i], tx), e2 = __fmaf_rn(dyh[i], tx, -p2);
        float sm, e3;
        two_sum(p1, p2, sm, e3);
        const float corr = (e1 + e2) + (e3 + __fmaf_rn(dxl[i], -ty, dyl[i] * tx));
        b[i] = __fadd_rn(sm, corr);
    }
    // 2. reference circle through hits 0, ib, ic (centre C in the chord frame)
    const float D = 2.f * __fmaf_rn(a[ib], b[ic], -__fmul_rn(b[ib], a[ic]));
    ok = ok && D != 0.f;
    const float uu = __fmaf_rn(a[ib], a[ib], b[ib] * b[ib]);
    const float vv = __fmaf_rn(a[ic], a[ic], b[ic] * b[ic]);
    const float iD = 1.f / D;
    const float Cx = (uu * b[ic] - vv * b[ib]) * iD, Cy = (vv * a[ib] - uu * a[ic]) * iD;
    const float R0 = sqrtf(__fmaf_rn(Cx, Cx, Cy * Cy));
    ok = ok && R0 < 1e7f;       // a nearly straight reference (pT above ~1e5 GeV): refitted
    const float sgn = D > 0.f ? 1.f : -1.f;
    // 3. outward residuals, arc lengths, z offsets from hit 0
    float sa[N], yr[N], zr[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i == 0) { sa[0] = yr[0] = zr[0] = 0.f; continue; }
        const float dx = a[i] - Cx, dy = b[i] - Cy;
        const float pw = __fmaf_rn(a[i], a[i] - 2.f * Cx, b[i] * (b[i] - 2.f * Cy));
        yr[i] = __fdividef(pw, sqrtf(__fmaf_rn(dx, dx, dy * dy)) + R0);
        const float cr = __fmaf_rn(Cy, a[i], -Cx * b[i]);                  // (-C) x (q - C)
        const float dt = __fmaf_rn(R0, R0, -__fmaf_rn(Cx, a[i], Cy * b[i]));  // (-C) . (q - C)
        sa[i] = R0 * arc_angle<true, float>(sgn * cr, dt);
        zr[i] = __fsub_rn(Z[i], Z[0]);
    }
    // 4. multiple scattering (float): one Highland angle per surface type
    const float cot0 = zr[ic] / sa[ic];
    const float sec2 = __fmaf_rn(cot0, cot0, 1.f);
    const float isec2 = 1.f / sec2;
    const float sec = sqrtf(sec2);
    const float a0 = 0.0136f / (float(kKpt * p.bfield) * R0 * sec);
    auto inv_th2 = [&](float path) {
        const float xx = float(p.x_over_x0) * path;
        const float th0 = a0 * sqrtf(xx) * (1.f + 0.038f * logf(xx));
        return 1.f / (th0 * th0);
    };
    bool any_disk = false;
#pragma unroll
    for (int i = 0; i < N; ++i) any_disk |= p.is_disk[L[i]] != 0;
    const float ib2 = inv_th2(sec);
    const float wz = float(p.w_z);
    float id2 = ib2, wdisk = wz;
    if (any_disk) {
        const float icot = 1.f / fabsf(cot0);
        id2 = inv_th2(sec * icot);
        const float iz = float(p.i_sz) * icot;             // disk: sigma_r = sigma_z |cot|
        wdisk = iz * iz;
    }
    // 5. rows of the normal equations (float values), matrices and solves in double
    double h[N], g[N], y64[N], z64[N], wT[N], wL[N], wkT[N], wkL[N];
    const double wrphi = p.w_rphi;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const float hf = i + 1 < N ? sa[i + 1] - sa[i] : 1.f;
        h[i] = hf;
        g[i] = 1.f / hf;
        y64[i] = yr[i];
        z64[i] = zr[i];
        const bool dk = p.is_disk[L[i]] != 0;
        wT[i] = wrphi;
        wL[i] = dk ? wdisk : wz;
        const float it2 = dk ? id2 : ib2;
        wkT[i] = it2 * isec2;                // kink variance th0^2 (1 + cot^2)
        wkL[i] = it2 * isec2 * isec2;        // kink variance th0^2 (1 + cot^2)^2
    }
#pragma unroll
    for (int j = 1; j + 1 < N; ++j)
        ok = ok && isfinite(wkT[j]) && isfinite(wkL[j]) && wkT[j] > 0.0 && wkL[j] > 0.0;
    double xT[N], xL[N], delta = 0.0, dummy, chi2T = 0.0, chi2L = 0.0;
    double cvT[6], cvL[3];
    if (!COV && !any_disk) {
        // every hit on a barrel layer: one measurement and one kink weight per view, the
        // geometry shared (the kink weights over the measurement weights; 1 / wz is sigma_z^2
        // to float rounding, far below the kink weights' own float rounding)
        const double lamT = wkT[1] * p.s2_rphi;
        const double lamL = wkL[1] * p.s2_z;
        // (the solve in double-float arithmetic)
        df64 hd[N], yd[N], zd[N], xTd[N], xLd[N], deltad, chi2d;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            hd[i] = df64(h[i]);
            yd[i] = df64(y64[i]);
            zd[i] = df64(z64[i]);
        }
        ok = ok && broken_line_pair<N, df64>(hd, yd, zd, df64(wrphi), df64(wL[0]), df64(lamT),
                                             df64(lamL), xTd, xLd, deltad, chi2d);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            xT[i] = double(xTd[i]);
            xL[i] = double(xLd[i]);
        }
        delta = double(deltad);
        chi2T = double(chi2d);
    } else {
        ok = ok && broken_line_n<N, true, double, COV>(h, y64, wT, wkT, xT, delta, chi2T, cvT) &&
             broken_line_n<N, false, double, COV>(h, z64, wL, wkL, xL, dummy, chi2L, cvL);
    }
    // 6. conversion in double: |C| and 1/|C| by two Newton steps from float (the fitted circle's
    // distance from the beam line needs its centre and radius consistent to ~1e-16 relative at
    // R0 ~ 1e7 cm), the chord direction to unit length, C turned back to the global frame
    const double Cxd = Cx, Cyd = Cy, r2 = Cxd * Cxd + Cyd * Cyd;
    double R0d = R0, iR0 = 1.f / R0;
    R0d += (r2 - R0d * R0d) * (0.5 * iR0);
    iR0 *= 2.0 - R0d * iR0;
    R0d += (r2 - R0d * R0d) * (0.5 * iR0);
    iR0 *= 2.0 - R0d * iR0;
    const double kappa = iR0 + delta;
    ok = ok && fabs(kappa) * 10.0 >= iR0;
    if (ok) {
        const double txd = tx, tyd = ty;
        const double un = rsqrt(txd * txd + tyd * tyd);
        const double ux = txd * un, uy = tyd * un;
        const double z0 = Z[0];
        const ConvGeom<double> G{iR0, Cxd * ux - Cyd * uy, Cxd * uy + Cyd * ux, double(sgn), g[0],
                                 h[0], double(X[0]), double(Y[0]), kKpt * p.bfield};
        ok = bl_convert<true, double>(G, xT[0], xT[1], delta, xL[0] + z0, xL[1] + z0, o);
        if (ok) {
            o.chi2 = chi2T + chi2L;
            o.status = 0;
            if constexpr (COV)
                bl_covariance<double>(G, xT[0], xT[1], delta, xL[0] + z0, xL[1] + z0, cvT, cvL,
                                      cov15);
        }
    }
    if (!ok) fit_refit64<N, COV>(X, Y, Z, L, p, o, cov15);
}

template <bool COV>
__device__ __forceinline__ void fit_track_split(int n, const float *X, const float *Y,
                                                const float *Z, const uint8_t *L,
                                                const DevParams &p, FitOut &o, double *cov15)
{
    switch (n) {
    case 3: fit_split_n<3, COV>(X, Y, Z, L, p, o, cov15); break;
    case 4: fit_split_n<4, COV>(X, Y, Z, L, p, o, cov15); break;
    case 5: fit_split_n<5, COV>(X, Y, Z, L, p, o, cov15); break;
    case 6: fit_split_n<6, COV>(X, Y, Z, L, p, o, cov15); break;
    default: o = FitOut{0, 0, 0, 0, 0, 0, 0, 4};
    }
}

// ---- Riemann fit (FP64) ----
// Smallest eigenpair of a symmetric 3 x 3 matrix: the eigenvalues in closed form (the
// trigonometric solution of the characteristic cubic of A - tr(A)/3), the eigenvector as the
// longest cross product of two rows of A - lambda I (orthogonal to both, so in the null space),
// then once more with the Rayleigh quotient of that vector as lambda.
__device__ __forceinline__ bool smallest_eigvec(const double (&A)[3][3], double (&v)[3])
{
    const double q = (A[0][0] + A[1][1] + A[2][2]) / 3.0;
    const double b00 = A[0][0] - q, b11 = A[1][1] - q, b22 = A[2][2] - q;
    const double p2 = b00 * b00 + b11 * b11 + b22 * b22 +
                      2.0 * (A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2]);
    const double p = sqrt(p2 / 6.0);
    if (!(p > 0.0)) return false;
    const double ip = 1.0 / p;
    const double c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip;
    const double c01 = A[0][1] * ip, c02 = A[0][2] * ip, c12 = A[1][2] * ip;
    const double det = c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) +
                       c02 * (c01 * c12 - c11 * c02);
    const double r = fmin(1.0, fmax(-1.0, 0.5 * det));
    const double phi = acos(r) / 3.0;
    double lam = q + 2.0 * p * cos(phi + 2.0943951023931957);   // the smallest root
    for (int it = 0; it < 2; ++it) {
        const double r0[3] = {A[0][0] - lam, A[0][1], A[0][2]};
        const double r1[3] = {A[1][0], A[1][1] - lam, A[1][2]};
        const double r2[3] = {A[2][0], A[2][1], A[2][2] - lam};
        auto cross = [](const double *a, const double *b, double *c) {
            c[0] = a[1] * b[2] - a[2] * b[1];
            c[1] = a[2] * b[0] - a[0] * b[2];
            c[2] = a[0] * b[1] - a[1] * b[0];
        };
        double x01[3], x02[3], x12[3];
        cross(r0, r1, x01);
        cross(r0, r2, x02);
        cross(r1, r2, x12);
        const double n01 = x01[0] * x01[0] + x01[1] * x01[1] + x01[2] * x01[2];
        const double n02 = x02[0] * x02[0] + x02[1] * x02[1] + x02[2] * x02[2];
        const double n12 = x12[0] * x12[0] + x12[1] * x12[1] + x12[2] * x12[2];
        const double *best = x01;
        double nb = n01;
        if (n02 > nb) { best = x02; nb = n02; }
        if (n12 > nb) { best = x12; nb = n12; }
        if (!(nb > 0.0)) return false;
        const double inv = rsqrt(nb);
        v[0] = best[0] * inv;
        v[1] = best[1] * inv;
        v[2] = best[2] * inv;
        double Av[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) Av[i] = A[i][0] * v[0] + A[i][1] * v[1] + A[i][2] * v[2];
        lam = v[0] * Av[0] + v[1] * Av[1] + v[2] * Av[2];
    }
    return true;
}

// Riemann fit of n hits (the same reading and output conventions as the broken line's
// conversion: orientation sgn, charge -sgn, arc lengths from hit 0, dxy = q (|C| - R)).
__device__ __noinline__ void riemann_fit(int n, const float *X, const float *Y, const float *Z,
                            const uint8_t *L, const DevParams &p, FitOut &o)
{
    o = FitOut{0, 0, 0, 0, 0, 0, 0, 0};
    if (n < 3 || n > kMaxHits) { o.status = 4; return; }
    const double w = 1.0 / (p.sigma_rphi * p.sigma_rphi);
    double P3[kMaxHits][3], m[3] = {0.0, 0.0, 0.0}, sw = 0.0;
    for (int i = 0; i < n; ++i) {
        const double x = X[i], y = Y[i];
        P3[i][0] = x;
        P3[i][1] = y;
        P3[i][2] = x * x + y * y;
#pragma unroll
        for (int k = 0; k < 3; ++k) m[k] += w * P3[i][k];
        sw += w;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) m[k] /= sw;
    double A[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (int i = 0; i < n; ++i) {
        const double d0 = P3[i][0] - m[0], d1 = P3[i][1] - m[1], d2 = P3[i][2] - m[2];
        A[0][0] += w * d0 * d0; A[0][1] += w * d0 * d1; A[0][2] += w * d0 * d2;
        A[1][1] += w * d1 * d1; A[1][2] += w * d1 * d2; A[2][2] += w * d2 * d2;
    }
    A[1][0] = A[0][1]; A[2][0] = A[0][2]; A[2][1] = A[1][2];
    double nv[3];
    if (!smallest_eigvec(A, nv) || nv[2] == 0.0) { o.status = 1; return; }
    const double c = -(nv[0] * m[0] + nv[1] * m[1] + nv[2] * m[2]);
    const double Cx = -nv[0] / (2.0 * nv[2]), Cy = -nv[1] / (2.0 * nv[2]);
    const double R2 = (nv[0] * nv[0] + nv[1] * nv[1] - 4.0 * c * nv[2]) / (4.0 * nv[2] * nv[2]);
    if (!(R2 > 0.0) || !isfinite(R2)) { o.status = 2; return; }
    const double R = sqrt(R2);
    const double ax = X[0] - Cx, ay = Y[0] - Cy;
    const double bx = X[n - 1] - Cx, by = Y[n - 1] - Cy;
    const double sgn = ax * by - ay * bx > 0.0 ? 1.0 : -1.0;
    const int q = sgn > 0.0 ? -1 : 1;
    double s[kMaxHits], wz[kMaxHits];
    for (int i = 0; i < n; ++i) {
        const double dx = X[i] - Cx, dy = Y[i] - Cy;
        s[i] = R * atan2(sgn * (ax * dy - ay * dx), ax * dx + ay * dy);
    }
    const double cot0 = (double(Z[n - 1]) - double(Z[0])) / (s[n - 1] - s[0]);
    double S0 = 0.0, S1 = 0.0, S2 = 0.0, T0 = 0.0, T1 = 0.0;
    for (int i = 0; i < n; ++i) {
        const double sz = p.is_disk[L[i]] ? p.sigma_z * fabs(cot0) : p.sigma_z;
        wz[i] = 1.0 / (sz * sz);
        S0 += wz[i];
        S1 += wz[i] * s[i];
        S2 += wz[i] * s[i] * s[i];
        T0 += wz[i] * double(Z[i]);
        T1 += wz[i] * s[i] * double(Z[i]);
    }
    const double det = S0 * S2 - S1 * S1;
    if (!(det > 0.0)) { o.status = 3; return; }
    const double cot = (S0 * T1 - S1 * T0) / det;
    const double z0 = (S2 * T0 - S1 * T1) / det;
    const double dC = sqrt(Cx * Cx + Cy * Cy);
    const double Px = Cx - R * Cx / dC, Py = Cy - R * Cy / dC;   // closest approach
    const double tpx = -sgn * (Py - Cy) / R, tpy = sgn * (Px - Cx) / R;
    const double s_pca = R * atan2(sgn * (ax * (Py - Cy) - ay * (Px - Cx)),
                                   ax * (Px - Cx) + ay * (Py - Cy));
    double chi2 = 0.0;
    for (int i = 0; i < n; ++i) {
        const double dx = X[i] - Cx, dy = Y[i] - Cy;
        const double d = sqrt(dx * dx + dy * dy) - R;
        const double e = double(Z[i]) - z0 - cot * s[i];
        chi2 += w * d * d + wz[i] * e * e;
    }
    o.pt = kKpt * p.bfield * R;
    o.phi = atan2(tpy, tpx);
    o.cot = cot;
    o.dxy = q * (dC - R);
    o.dz = z0 + cot * s_pca;
    o.chi2 = chi2;
    o.q = (int8_t)q;
    o.status = 0;
}

template <bool COV, bool SPLIT>
__device__ __forceinline__ void fit_dispatch(int n, const float *X, const float *Y,
                                             const float *Z, const uint8_t *L,
                                             const DevParams &p, FitOut &o, double *cov15)
{
    if constexpr (SPLIT) {
        fit_track_split<COV>(n, X, Y, Z, L, p, o, cov15);
        return;
    }
    if (p.fit_mode == FIT_RIEMANN) {
        riemann_fit(n, X, Y, Z, L, p, o);
        if constexpr (COV) {
#pragma unroll
            for (int k = 0; k < 15; ++k) cov15[k] = __longlong_as_double(0x7FF8000000000000LL);
        }
        return;
    }
    if (p.fit_mode == FIT_MIXED) fit_track<double, double, true, COV>(n, X, Y, Z, L, p, o, cov15);
    else if (p.fit_mode == FIT_FP32) fit_track<float, float, false, COV>(n, X, Y, Z, L, p, o, cov15);
    else fit_track<double, double, false, COV>(n, X, Y, Z, L, p, o, cov15);
}

// Selection rank of a good track for shared-hit cleaning: more hits first, then smaller
// chi2/ndof.  A 64-bit key ordered like that rank: 7 - n in the top bits, then the bits of the
// non-negative double chi2/ndof (ordered like its value) without their last four.
__device__ __forceinline__ unsigned long long rank_key(int n, double chi2_ndof)
{
    return ((unsigned long long)(7 - n) << 60) |
           ((unsigned long long)__double_as_longlong(chi2_ndof) >> 4);
}

__device__ __forceinline__ double chi2_ndof(double chi2, int n)
{
    return chi2 / (double)(2 * n - 5 > 1 ? 2 * n - 5 : 1);
}

// One thread per output track: the kept ntuplets are listed per event in output order, and the
// number of outputs is read on the device, so no thread is spent on unused capacity.  After the
// fit, the selection cuts give the track's quality; with shared-hit cleaning a good track offers
// its rank key to each of its hits (the smallest key of a hit wins, k_keep reads them).
template <bool COV, bool SPLIT>
__global__ void __launch_bounds__(256, 2) k_fit(DevBatch b, DevParams p)
{
    const uint32_t n_out = b.out_evt[b.E];
    for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out;
         o += gridDim.x * blockDim.x) {
        const uint32_t e = find_event(b.out_evt, b.E, o);
        const uint32_t t = b.tup_list[b.tup_off[e] + (o - b.out_evt[e])];
        const int n = b.tup_n[t];
        float X[kMaxHits], Y[kMaxHits], Z[kMaxHits];
        uint8_t L[kMaxHits];
#pragma unroll
        for (int h = 0; h < kMaxHits; ++h) {
            const uint32_t pos = b.tup_hits[(size_t)t * kMaxHits + h];
            if (h < n && PXR_IN(b, e, pos, b.N)) {
                const float4 v = b.hs[pos];
                const uint32_t meta = b.hmeta[pos];
                X[h] = v.x; Y[h] = v.y; Z[h] = v.z;
                L[h] = (uint8_t)(meta >> kLocalBits);
                b.o_hits[(size_t)o * kMaxHits + h] = meta & kLocalMask;
            } else {
                X[h] = Y[h] = Z[h] = 0.f;
                L[h] = 0;
                b.o_hits[(size_t)o * kMaxHits + h] = kNone;
            }
        }
        FitOut f;
        double cv[COV ? 15 : 1];
        fit_dispatch<COV, SPLIT>(n, X, Y, Z, L, p, f, cv);
        if constexpr (COV) {
#pragma unroll
            for (int k = 0; k < 15; ++k)
                b.o_cov[(size_t)o * 15 + k] =
                    f.status == 0 ? cv[k] : __longlong_as_double(0x7FF8000000000000LL);
        }
        b.o_nh[o] = (uint8_t)n;
        b.o_pt[o] = f.pt; b.o_phi[o] = f.phi; b.o_cot[o] = f.cot;
        b.o_dxy[o] = f.dxy; b.o_dz[o] = f.dz; b.o_chi2[o] = f.chi2;
        b.o_q[o] = f.q; b.o_status[o] = f.status;
        // (the FP64 division only when a cut or the ranking needs chi2/ndof)
        const bool need_r = p.chi2_max > 0.0 || p.clean;
        const double r = need_r ? chi2_ndof(f.chi2, n) : 0.0;
        const bool good = f.status == 0 && isfinite(f.chi2) &&
                          (p.pt_min <= 0.0 || f.pt >= p.pt_min) &&
                          (p.chi2_max <= 0.0 || r <= p.chi2_max);
        b.o_ql[o] = good ? (uint8_t)(kQGood | (p.clean ? 0u : kQKept)) : (uint8_t)0;
        if (good && p.clean) {
            const unsigned long long key = rank_key(n, r);
            const uint32_t h0 = b.hit_off[e];
            for (int h = 0; h < n; ++h)          // (the hit indices this thread wrote above)
                atomicMin(&b.best[h0 + b.o_hits[(size_t)o * kMaxHits + h]], key);
        }
    }
}

// Shared-hit cleaning, after every good track has offered its key: a good track is kept when no
// hit of it carries a smaller key (a better-ranked good track sharing the hit).
__global__ void __launch_bounds__(256) k_keep(DevBatch b)
{
    const uint32_t n_out = b.out_evt[b.E];
    for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out;
         o += gridDim.x * blockDim.x) {
        const uint8_t ql = b.o_ql[o];
        if (!(ql & kQGood)) continue;
        const uint32_t e = find_event(b.out_evt, b.E, o);
        const int n = b.o_nh[o];
        const unsigned long long key = rank_key(n, chi2_ndof(b.o_chi2[o], n));
        const uint32_t h0 = b.hit_off[e];
        bool kept = true;
        for (int h = 0; h < n; ++h)
            kept &= b.best[h0 + b.o_hits[(size_t)o * kMaxHits + h]] >= key;
        if (kept) b.o_ql[o] = (uint8_t)(ql | kQKept);
    }
}

void launch_fit(const DevBatch &b, const DevParams &p, uint32_t total, cudaStream_t s, int sms)
{
    // a few hundred fits are bound by the FP64 pipe of the SMs they run on: small batches take
    // smaller blocks, so that their tracks spread over more SMs
    uint32_t tpb = p.block_threads[5];
    if (tpb == 0) {
        tpb = 32;
        while (tpb < 256 && (uint64_t)tpb * sms < total) tpb *= 2;
    }
    uint64_t blocks = ((uint64_t)total + tpb - 1) / tpb;
    uint64_t cap = (uint64_t)sms * p.grid_per_sm[5] * (256 / tpb);
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    const bool split = p.fit_mode == FIT_SPLIT;
    if (p.cov) {
        if (split) k_fit<true, true><<<(unsigned)blocks, tpb, 0, s>>>(b, p);
        else k_fit<true, false><<<(unsigned)blocks, tpb, 0, s>>>(b, p);
    } else {
        if (split) k_fit<false, true><<<(unsigned)blocks, tpb, 0, s>>>(b, p);
        else k_fit<false, false><<<(unsigned)blocks, tpb, 0, s>>>(b, p);
    }
}

void launch_keep(const DevBatch &b, const DevParams &p, uint32_t total, cudaStream_t s, int sms)
{
    uint64_t blocks = ((uint64_t)total + 255) / 256;
    const uint64_t cap = (uint64_t)sms * p.grid_per_sm[5];     // the fit stage's cap
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    k_keep<<<(unsigned)blocks, 256, 0, s>>>(b);
}

// ---- primary vertices ----
constexpr int kVtxMax = 8192;      // kept tracks per event the vertex finder takes (more: flagged)
constexpr int kVtxThreads = 512;

// One CTA per event.  The kept tracks with a finite dz are gathered into shared memory (dz, pT^2,
// output slot) and sorted by (dz, output slot) with a bitonic network; a sorted track starts a new cluster when
// its dz exceeds the previous one's by more than the gap.  Each cluster start counts its members;
// clusters of at least vtx_min tracks become vertices (a block-wide scan gives their cluster-
// order index).  Each vertex's start sums its members in sorted order (mean dz, the standard
// error of the mean, sum pT^2), the records go to the event's vertex arrays, and each record is
// then moved to its rank by (sum pT^2 descending, z ascending) and stamped on its tracks.
__global__ void __launch_bounds__(kVtxThreads) k_vertices(DevBatch b, DevParams p)
{
    extern __shared__ unsigned char vsm[];
    double *sz = reinterpret_cast<double *>(vsm);                 // [kVtxMax] dz
    double *sp = sz + kVtxMax;                                    // [kVtxMax] pT^2 (sorted along)
    uint32_t *si = reinterpret_cast<uint32_t *>(sp + kVtxMax);    // [kVtxMax] output slot
    __shared__ uint32_t s_m, s_wsum[kVtxThreads / 32];
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    for (uint32_t e = blockIdx.x; e < b.E; e += gridDim.x) {
        const uint32_t a = b.out_evt[e], n = b.out_evt[e + 1] - a;
        for (uint32_t t = tid; t < n; t += nt) b.o_vtx[a + t] = -1;
        if (tid == 0) s_m = 0;
        __syncthreads();
        for (uint32_t t = tid; t < n; t += nt) {
            const double dz = b.o_dz[a + t];
            if ((b.o_ql[a + t] & kQKept) && isfinite(dz)) {
                const uint32_t k = atomicAdd(&s_m, 1u);
                if (k < (uint32_t)kVtxMax) {
                    const double pt = b.o_pt[a + t];
                    sz[k] = dz;
                    sp[k] = pt * pt;
                    si[k] = t;
                }
            }
        }
        __syncthreads();
        const uint32_t m = s_m;
        if (m > (uint32_t)kVtxMax) {                   // uniform: too many tracks, no vertices
            if (tid == 0) {
                b.cnt[C_VERTS * b.E + e] = 0;
                atomicOr(&b.cnt[C_FLAGS * b.E + e], F_VERTS);
            }
            __syncthreads();
            continue;
        }
        uint32_t P2 = 1;
        while (P2 < m) P2 <<= 1;
        for (uint32_t k = m + tid; k < P2; k += nt) {
            sz[k] = __longlong_as_double(0x7FF0000000000000LL);   // +inf after every track
            si[k] = 0xFFFFFFFFu;
        }
        __syncthreads();
        for (uint32_t size = 2; size <= P2; size <<= 1)
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (uint32_t i = tid; i < P2; i += nt) {
                    const uint32_t j = i ^ stride;
                    if (j > i) {
                        const bool asc = (i & size) == 0;
                        const bool jl = sz[j] < sz[i] || (sz[j] == sz[i] && si[j] < si[i]);
                        if (asc == jl) {
                            const double tz = sz[i]; sz[i] = sz[j]; sz[j] = tz;
                            const double tp = sp[i]; sp[i] = sp[j]; sp[j] = tp;
                            const uint32_t ti = si[i]; si[i] = si[j]; si[j] = ti;
                        }
                    }
                }
                __syncthreads();
            }
        // each thread owns a run of consecutive sorted positions; a position is a vertex start
        // when it starts a cluster of at least vtx_min tracks
        const uint32_t per = (m + nt - 1) / nt;
        const uint32_t k0 = min(m, tid * per), k1 = min(m, k0 + per);
        auto starts = [&](uint32_t k) { return k == 0 || sz[k] - sz[k - 1] > p.vtx_gap; };
        auto members = [&](uint32_t k) {
            uint32_t c = 1;
            while (k + c < m && !starts(k + c)) ++c;
            return c;
        };
        uint32_t mine = 0;
        for (uint32_t k = k0; k < k1; ++k)
            if (starts(k) && members(k) >= p.vtx_min) ++mine;
        // block-wide exclusive scan of the counts
        const uint32_t lane = tid & 31u, wid = tid >> 5;
        uint32_t incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += t;
        }
        if (lane == 31) s_wsum[wid] = incl;
        __syncthreads();
        uint32_t before = 0, nv = 0;
        for (uint32_t w = 0; w < nt / 32; ++w) {
            if (w < wid) before += s_wsum[w];
            nv += s_wsum[w];
        }
        uint32_t vi = before + incl - mine;
        // the vertex records, in cluster order, at the event's vertex arrays
        for (uint32_t k = k0; k < k1; ++k) {
            if (!starts(k)) continue;
            const uint32_t c = members(k);
            if (c < p.vtx_min) continue;
            double sum = 0.0, pt2 = 0.0;
            for (uint32_t q = 0; q < c; ++q) {
                sum += sz[k + q];
                pt2 += sp[k + q];
            }
            const double z = sum / (double)c;
            double ss = 0.0;
            for (uint32_t q = 0; q < c; ++q) ss += (sz[k + q] - z) * (sz[k + q] - z);
            b.v_z[a + vi] = z;
            b.v_err[a + vi] = c > 1 ? sqrt(ss / ((double)c * (double)(c - 1))) : 0.0;
            b.v_pt2[a + vi] = pt2;
            b.v_n[a + vi] = k;                          // (the start, until the final pass)
            ++vi;
        }
        __syncthreads();
        // ranks: sum pT^2 descending, then z ascending (vertex records owned per thread)
        constexpr int kOwn = kVtxMax / kVtxThreads;   // records per thread at most (vtx_min >= 2)
        double oz[kOwn], oe[kOwn], op[kOwn];
        uint32_t ok_[kOwn], orank[kOwn];
        int own = 0;
        for (uint32_t v = tid; v < nv && own < kOwn; v += nt, ++own) {
            oz[own] = b.v_z[a + v];
            oe[own] = b.v_err[a + v];
            op[own] = b.v_pt2[a + v];
            ok_[own] = b.v_n[a + v];
            uint32_t r = 0;
            for (uint32_t u = 0; u < nv; ++u) {
                const double pu = b.v_pt2[a + u], zu = b.v_z[a + u];
                r += pu > op[own] || (pu == op[own] && (zu < oz[own] || (zu == oz[own] && u < v)));
            }
            orank[own] = r;
        }
        __syncthreads();
        for (int q = 0; q < own; ++q) {
            const uint32_t r = orank[q], k = ok_[q];
            const uint32_t c = members(k);
            b.v_z[a + r] = oz[q];
            b.v_err[a + r] = oe[q];
            b.v_pt2[a + r] = op[q];
            b.v_n[a + r] = c;
            for (uint32_t t = 0; t < c; ++t) b.o_vtx[a + si[k + t]] = (int32_t)r;
        }
        if (tid == 0) b.cnt[C_VERTS * b.E + e] = nv;
        __syncthreads();
    }
}

cudaError_t init_fit_kernels()
{
    return cudaFuncSetAttribute(k_vertices, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kVtxMax * (int)(2 * sizeof(double) + sizeof(uint32_t)));
}

void launch_vertices(const DevBatch &b, const DevParams &p, cudaStream_t s, int sms)
{
    if (b.E == 0) return;
    const size_t smem = (size_t)kVtxMax * (2 * sizeof(double) + sizeof(uint32_t));
    const uint32_t grid = b.E < (uint32_t)sms * 2 ? b.E : (uint32_t)sms * 2;
    k_vertices<<<grid, kVtxThreads, smem, s>>>(b, p);
}

// Fit-only path: m ntuplets given directly.
template <bool SPLIT>
__global__ void __launch_bounds__(128, 4) k_fit_batch(uint32_t m, const uint8_t *nh, const float *x,
                                                   const float *y, const float *z,
                                                   const uint16_t *layer, uint32_t stride,
                                                   DevParams p, double *pt, double *phi,
                                                   double *cot, double *dxy, double *dz,
                                                   double *chi2, int8_t *q, int8_t *status)
{
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int n = nh[t];
        float X[kMaxHits], Y[kMaxHits], Z[kMaxHits];
        uint8_t L[kMaxHits];
        for (int h = 0; h < kMaxHits; ++h) {
            if (h < n && h < (int)stride) {
                const size_t k = (size_t)t * stride + h;
                X[h] = x[k]; Y[h] = y[k]; Z[h] = z[k];
                const uint16_t l = layer[k];
                L[h] = (uint8_t)(l < p.n_layers ? l : 0);
            } else {
                X[h] = Y[h] = Z[h] = 0.f;
                L[h] = 0;
            }
        }
        FitOut f;
        fit_dispatch<false, SPLIT>(n <= (int)stride ? n : 0, X, Y, Z, L, p, f, nullptr);
        pt[t] = f.pt; phi[t] = f.phi; cot[t] = f.cot; dxy[t] = f.dxy; dz[t] = f.dz;
        chi2[t] = f.chi2; q[t] = f.q; status[t] = f.status;
    }
}

void launch_fit_batch(uint32_t m, const uint8_t *nh, const float *x, const float *y,
                      const float *z, const uint16_t *layer, uint32_t stride, const DevParams &p,
                      double *pt, double *phi, double *cot, double *dxy, double *dz, double *chi2,
                      int8_t *q, int8_t *status, cudaStream_t s, int sms)
{
    uint64_t blocks = ((uint64_t)m + 127) / 128;
    uint64_t cap = (uint64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    if (p.fit_mode == FIT_SPLIT)
        k_fit_batch<true><<<(unsigned)blocks, 128, 0, s>>>(m, nh, x, y, z, layer, stride, p, pt,
                                                           phi, cot, dxy, dz, chi2, q, status);
    else
        k_fit_batch<false><<<(unsigned)blocks, 128, 0, s>>>(m, nh, x, y, z, layer, stride, p, pt,
                                                            phi, cot, dxy, dz, chi2, q, status);
}

}  // namespace pxr
