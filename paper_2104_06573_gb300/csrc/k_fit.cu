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
//     (z_i); the normal equations are a pentadiagonal block bordered (transverse) by the
//     curvature row, solved by a banded Cholesky and the Schur complement of the border;
//  5. fitted circle at hit 0 and its point of closest approach to the z axis.
// Precision modes: FP64 (all steps double), MIXED (arithmetic double, transcendentals float:
// the normal matrices mix kink weights up to ~1e14 with measurement weights ~1e6, which float
// assembly cannot hold), FP32 (all float).  The hit count is a template parameter, so every
// array lives in registers.
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

// Symmetric positive definite pentadiagonal matrix (diagonal d0, first and second
// super-diagonals d1, d2) factored as L L^T in place: d1, d2 receive L's sub-diagonals and d0
// the reciprocals of L's diagonal (so the solves multiply instead of divide).
template <int N, typename T>
__device__ __forceinline__ bool band_factor(T (&d0)[N], T (&d1)[N], T (&d2)[N])
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T s = d0[i];
        if (i >= 1) s -= d1[i - 1] * d1[i - 1];
        if (i >= 2) s -= d2[i - 2] * d2[i - 2];
        if (!(s > T(0))) return false;
        const T il = rsqrt_t(s);
        d0[i] = il;
        if (i + 1 < N) {
            T t = d1[i];
            if (i >= 1) t -= d2[i - 1] * d1[i - 1];
            d1[i] = t * il;
        }
        if (i + 2 < N) d2[i] = d2[i] * il;
    }
    return true;
}

// Solve (L L^T) x = b with the factor of band_factor (il: reciprocal diagonal).
template <int N, typename T>
__device__ __forceinline__ void band_solve(const T (&il)[N], const T (&l1)[N], const T (&l2)[N],
                                           const T (&b)[N], T (&x)[N])
{
    T y[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T t = b[i];
        if (i >= 1) t -= l1[i - 1] * y[i - 1];
        if (i >= 2) t -= l2[i - 2] * y[i - 2];
        y[i] = t * il[i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        T t = y[i];
        if (i + 1 < N) t -= l1[i] * x[i + 1];
        if (i + 2 < N) t -= l2[i] * x[i + 2];
        x[i] = t * il[i];
    }
}

// Broken line over N points: measurements meas (weights w), kinks at the inner points j with
// weights wk[j] (reciprocal variances), and (CURV) one curvature unknown.  g[i] = 1/(s[i+1]-s[i])
// and h[i] = s[i+1]-s[i].  Normal equations: a pentadiagonal block for the offsets (each kink
// couples three neighbours) bordered by the curvature row; the border is eliminated through the
// Schur complement.  Returns the offsets x, the curvature correction and the chi2 at the minimum;
// with CV, also the covariance of (x_0, x_1[, delta]) (the corresponding block of the inverse
// normal matrix: cv = c00, c01, c11 and, with CURV, c0d, c1d, cdd).
template <int N, bool CURV, typename T, bool CV = false>
__device__ __forceinline__ bool broken_line_n(const T (&g)[N], const T (&h)[N], const T (&meas)[N],
                                              const T (&w)[N], const T (&wk)[N], T (&x)[N],
                                              T &delta, T &chi2, T *cv = nullptr)
{
    T d0[N], d1[N], d2[N], c[N], b[N];
    T dd = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        d0[i] = w[i];
        d1[i] = T(0);
        d2[i] = T(0);
        c[i] = T(0);
        b[i] = w[i] * meas[i];
    }
#pragma unroll
    for (int j = 1; j + 1 < N; ++j) {
        const T g0 = g[j - 1], g2 = g[j], g1 = -g0 - g2;
        const T k = wk[j];
        d0[j - 1] += k * g0 * g0;
        d0[j] += k * g1 * g1;
        d0[j + 1] += k * g2 * g2;
        d1[j - 1] += k * g0 * g1;
        d1[j] += k * g1 * g2;
        d2[j - 1] += k * g0 * g2;
        if (CURV) {
            const T gd = T(0.5) * (h[j - 1] + h[j]);
            c[j - 1] += k * g0 * gd;
            c[j] += k * g1 * gd;
            c[j + 1] += k * g2 * gd;
            dd += k * gd * gd;
        }
    }
    if (!band_factor<N, T>(d0, d1, d2)) return false;
    band_solve<N, T>(d0, d1, d2, b, x);
    delta = T(0);
    T z[N], schur = T(1);
    if (CURV) {
        band_solve<N, T>(d0, d1, d2, c, z);
        T cy = T(0), cz = T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            cy += c[i] * x[i];
            cz += c[i] * z[i];
        }
        schur = dd - cz;
        if (!(schur > T(0))) return false;
        delta = -cy / schur;
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] -= z[i] * delta;
    }
    if constexpr (CV) {
        // columns 0 and 1 of the inverse of the pentadiagonal block; the bordered inverse adds
        // z z^T / S to it, with -z / S and 1 / S for the curvature (S the Schur complement)
        T e[N], y0[N], y1[N];
#pragma unroll
        for (int i = 0; i < N; ++i) e[i] = i == 0 ? T(1) : T(0);
        band_solve<N, T>(d0, d1, d2, e, y0);
#pragma unroll
        for (int i = 0; i < N; ++i) e[i] = i == 1 ? T(1) : T(0);
        band_solve<N, T>(d0, d1, d2, e, y1);
        cv[0] = y0[0];
        cv[1] = y0[1];
        cv[2] = y1[1];
        if (CURV) {
            const T is = T(1) / schur;
            cv[0] += z[0] * z[0] * is;
            cv[1] += z[0] * z[1] * is;
            cv[2] += z[1] * z[1] * is;
            cv[3] = -z[0] * is;
            cv[4] = -z[1] * is;
            cv[5] = is;
        }
    }
    T c2 = T(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const T r = meas[i] - x[i];
        c2 += w[i] * r * r;
    }
#pragma unroll
    for (int j = 1; j + 1 < N; ++j) {
        T beta = (x[j + 1] - x[j]) * g[j] - (x[j] - x[j - 1]) * g[j - 1];
        if (CURV) beta += T(0.5) * (h[j - 1] + h[j]) * delta;
        c2 += beta * beta * wk[j];
    }
    chi2 = c2;
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

// TC: prefit + residuals + arc lengths; T: everything else (scattering, solves, conversion);
// FT: float transcendentals (angles and logarithms need ~1e-7 relative, far inside the
// tolerances).  Divisions and square roots are shared where the method allows (one reciprocal
// per arc-length step, one scattering angle per surface type, reciprocal Cholesky pivots): they
// are the costly operations of the double-precision path.
template <int N, typename TC, typename T, bool FT, bool COV>
__device__ void fit_n(const float *X, const float *Y, const float *Z, const uint8_t *L,
                      const DevParams &p, FitOut &o, double *cov15)
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
    if (!broken_line_n<N, true, T, COV>(g, h, yr, wT, wkT, xT, delta, chi2T, cvT) ||
        !broken_line_n<N, false, T, COV>(g, h, z, wL, wkL, xL, dummy, chi2L, cvL)) {
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
    if constexpr (COV) {
        // covariance of (q/pT, phi, cot, dxy, dz): the fitted values' covariance (the blocks of
        // the inverse normal matrices; the two broken lines are independent) through the
        // conversion's Jacobian (forward-mode derivatives in FP64)
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
        q0[0] = D5(double(xT[0]));
        q0[1] = D5(double(xT[1]));
        q0[2] = D5(double(delta));
        q0[3] = D5(double(xL[0]));
        q0[4] = D5(double(xL[1]));
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

template <bool COV>
__device__ __forceinline__ void fit_dispatch(int n, const float *X, const float *Y,
                                             const float *Z, const uint8_t *L,
                                             const DevParams &p, FitOut &o, double *cov15)
{
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
template <bool COV>
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
            if (h < n) {
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
        fit_dispatch<COV>(n, X, Y, Z, L, p, f, cv);
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
    uint32_t tpb = 32;
    while (tpb < 256 && (uint64_t)tpb * sms < total) tpb *= 2;
    uint64_t blocks = ((uint64_t)total + tpb - 1) / tpb;
    uint64_t cap = (uint64_t)sms * p.grid_per_sm[5] * (256 / tpb);
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    if (p.cov) k_fit<true><<<(unsigned)blocks, tpb, 0, s>>>(b, p);
    else k_fit<false><<<(unsigned)blocks, tpb, 0, s>>>(b, p);
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
__global__ void __launch_bounds__(128) k_fit_batch(uint32_t m, const uint8_t *nh, const float *x,
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
        fit_dispatch<false>(n <= (int)stride ? n : 0, X, Y, Z, L, p, f, nullptr);
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
    k_fit_batch<<<(unsigned)blocks, 128, 0, s>>>(m, nh, x, y, z, layer, stride, p, pt, phi, cot,
                                                 dxy, dz, chi2, q, status);
}

}  // namespace pxr
