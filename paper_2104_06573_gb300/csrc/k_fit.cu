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
//     (z_i), normal equations solved by Cholesky;
//  5. fitted circle at hit 0 and its point of closest approach to the z axis.
// Precision modes: FP64 (all steps double), MIXED (arithmetic double, transcendentals float:
// the normal matrices mix kink weights up to ~1e14 with measurement weights ~1e6, which float
// assembly cannot hold), FP32 (all float).
#include "pxr_dev.cuh"

namespace pxr {

constexpr double kKpt = 0.299792458e-2;   // pT [GeV] = K B [T] R [cm]
constexpr int kM = kMaxHits + 1;

template <typename T>
__device__ __forceinline__ T sqrt_t(T v) { return sqrt(v); }
template <>
__device__ __forceinline__ float sqrt_t<float>(float v) { return sqrtf(v); }

// Dense Cholesky of the m x m SPD matrix A (row-major, m <= kM), then two triangular solves.
template <typename T>
__device__ __forceinline__ bool chol_solve(int m, T *A, const T *b, T *x)
{
    for (int j = 0; j < m; ++j) {
        T s = A[j * kM + j];
        for (int k = 0; k < j; ++k) s -= A[j * kM + k] * A[j * kM + k];
        if (!(s > T(0))) return false;
        const T d = sqrt_t(s);
        A[j * kM + j] = d;
        for (int i = j + 1; i < m; ++i) {
            T t = A[i * kM + j];
            for (int k = 0; k < j; ++k) t -= A[i * kM + k] * A[j * kM + k];
            A[i * kM + j] = t / d;
        }
    }
    T y[kM];
    for (int i = 0; i < m; ++i) {
        T t = b[i];
        for (int k = 0; k < i; ++k) t -= A[i * kM + k] * y[k];
        y[i] = t / A[i * kM + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        T t = y[i];
        for (int k = i + 1; k < m; ++k) t -= A[k * kM + i] * x[k];
        x[i] = t / A[i * kM + i];
    }
    return true;
}

// Normal equations of the broken line: measurements meas (weights w), kinks at inner points with
// variance kv, optional curvature unknown at index n.  Assembled in TB, solved in TS.
template <typename TB, typename TS>
__device__ __forceinline__ bool broken_line(int n, const TB *s, const TB *meas, const TB *w,
                                            const TB *kv, bool curv, TS *x, TS &chi2)
{
    const int m = n + (curv ? 1 : 0);
    TB A[kM * kM];
    TB bb[kM];
    for (int r = 0; r < m; ++r) {
        bb[r] = TB(0);
        for (int c = 0; c < m; ++c) A[r * kM + c] = TB(0);
    }
    for (int i = 0; i < n; ++i) {
        A[i * kM + i] += w[i];
        bb[i] += w[i] * meas[i];
    }
    for (int j = 1; j + 1 < n; ++j) {
        const TB ds0 = s[j] - s[j - 1], ds1 = s[j + 1] - s[j];
        const TB wk = TB(1) / kv[j];
        const int idx[4] = {j - 1, j, j + 1, n};
        const TB g[4] = {TB(1) / ds0, -TB(1) / ds0 - TB(1) / ds1, TB(1) / ds1,
                         curv ? TB(0.5) * (ds0 + ds1) : TB(0)};
        const int q = curv ? 4 : 3;
        for (int r = 0; r < q; ++r)
            for (int c = 0; c < q; ++c) A[idx[r] * kM + idx[c]] += wk * g[r] * g[c];
    }
    TS As[kM * kM], bs[kM];
    for (int r = 0; r < m; ++r) {
        bs[r] = TS(bb[r]);
        for (int c = 0; c < m; ++c) As[r * kM + c] = TS(A[r * kM + c]);
    }
    if (!chol_solve<TS>(m, As, bs, x)) return false;
    TS c2 = TS(0);
    for (int i = 0; i < n; ++i) {
        const TS r = TS(meas[i]) - x[i];
        c2 += TS(w[i]) * r * r;
    }
    for (int j = 1; j + 1 < n; ++j) {
        const TS ds0 = TS(s[j]) - TS(s[j - 1]), ds1 = TS(s[j + 1]) - TS(s[j]);
        TS beta = (x[j + 1] - x[j]) / ds1 - (x[j] - x[j - 1]) / ds0;
        if (curv) beta += TS(0.5) * (ds0 + ds1) * x[n];
        c2 += beta * beta / TS(kv[j]);
    }
    chi2 = c2;
    return true;
}

struct FitOut {
    double pt, phi, cot, dxy, dz, chi2;
    int8_t q, status;
};

// Transcendentals in float (FT = true) or in the argument's own type.
template <bool FT, typename T>
__device__ __forceinline__ T atan2_t(T y, T x) { return FT ? T(atan2f(float(y), float(x))) : atan2(y, x); }
template <bool FT, typename T>
__device__ __forceinline__ T log_t(T v) { return FT ? T(logf(float(v))) : log(v); }

// TC: prefit + residuals; TB: scattering + assembly; TS: solves + conversion; FT: float
// transcendentals (angles and logarithms need ~1e-7 relative, far inside the tolerances).
template <typename TC, typename TB, typename TS, bool FT>
__device__ void fit_track(int n, const float *X, const float *Y, const float *Z,
                          const uint8_t *L, const DevParams &p, FitOut &o)
{
    o = FitOut{0, 0, 0, 0, 0, 0, 0, 0};
    if (n < 3 || n > kMaxHits) { o.status = 4; return; }
    TC px[kMaxHits], py[kMaxHits];
    const TC x0 = TC(X[0]), y0 = TC(Y[0]);
    for (int i = 0; i < n; ++i) { px[i] = TC(X[i]) - x0; py[i] = TC(Y[i]) - y0; }
    const int ib = n / 2, ic = n - 1;
    const TC ux = px[ib], uy = py[ib], vx = px[ic], vy = py[ic];
    const TC D = TC(2) * (ux * vy - uy * vx);
    if (D == TC(0)) { o.status = 1; return; }
    const TC uu = ux * ux + uy * uy, vv = vx * vx + vy * vy;
    const TC Cx = (uu * vy - vv * uy) / D, Cy = (vv * ux - uu * vx) / D;
    const TC R0 = sqrt_t(Cx * Cx + Cy * Cy);
    const TC sgn = D > TC(0) ? TC(1) : TC(-1);

    TB s[kMaxHits], yr[kMaxHits], z[kMaxHits];
    for (int i = 0; i < n; ++i) {
        const TC dx = px[i] - Cx, dy = py[i] - Cy;
        const TC pw = (px[i] * px[i] + py[i] * py[i]) - TC(2) * (px[i] * Cx + py[i] * Cy);
        yr[i] = TB(pw / (sqrt_t(dx * dx + dy * dy) + R0));
        const TC cr = -Cx * dy + Cy * dx;
        const TC dt = -Cx * dx - Cy * dy;
        s[i] = TB(R0 * atan2_t<FT>(sgn * cr, dt));
        z[i] = TB(Z[i]);
    }

    // multiple scattering
    const TB cot0 = (z[ic] - z[0]) / (s[ic] - s[0]);
    const TB sec2 = TB(1) + cot0 * cot0;
    const TB pmom = TB(kKpt * p.bfield) * TB(R0) * sqrt_t(sec2);
    TB kvT[kMaxHits], kvL[kMaxHits], wT[kMaxHits], wL[kMaxHits];
    const TB wrphi = TB(1.0 / (p.sigma_rphi * p.sigma_rphi));
    const TB wz = TB(1.0 / (p.sigma_z * p.sigma_z));
    for (int i = 0; i < n; ++i) {
        kvT[i] = TB(1);
        kvL[i] = TB(1);
        wT[i] = wrphi;
        if (p.is_disk[L[i]]) {
            const TB sz = TB(p.sigma_z) * fabs(cot0);
            wL[i] = TB(1) / (sz * sz);
        } else {
            wL[i] = wz;
        }
    }
    for (int j = 1; j + 1 < n; ++j) {
        const TB path = p.is_disk[L[j]] ? sqrt_t(sec2) / fabs(cot0) : sqrt_t(sec2);
        const TB xx = TB(p.x_over_x0) * path;
        const TB th0 = (TB(0.0136) / pmom) * sqrt_t(xx) * (TB(1) + TB(0.038) * log_t<FT>(xx));
        const TB th2 = th0 * th0;
        kvT[j] = th2 * sec2;
        kvL[j] = th2 * sec2 * sec2;
        if (!(kvT[j] > TB(0)) || !(kvL[j] > TB(0))) { o.status = 4; return; }
    }

    TS xT[kM], xL[kM];
    TS chi2T, chi2L;
    if (!broken_line<TB, TS>(n, s, yr, wT, kvT, true, xT, chi2T) ||
        !broken_line<TB, TS>(n, s, z, wL, kvL, false, xL, chi2L)) {
        o.status = 3;
        return;
    }

    // conversion to the point of closest approach
    const TS delta = xT[n];
    const TS R0s = TS(R0);
    const TS kappa = TS(1) / R0s + delta;
    if (kappa == TS(0) || !isfinite(kappa)) { o.status = 2; return; }
    const TS R = TS(1) / fabs(kappa);
    const TS sgs = TS(sgn);
    const TS sgf = kappa > TS(0) ? sgs : -sgs;
    const TS ds0 = TS(s[1]) - TS(s[0]);
    const TS alpha = (xT[1] - xT[0]) / ds0 + TS(0.5) * delta * ds0;
    const TS nx = -TS(Cx) / R0s, ny = -TS(Cy) / R0s;
    const TS tx = -sgs * ny, ty = sgs * nx;
    TS ca, sa;
    if constexpr (FT) {
        // cos of a small angle rounds to 1 in float; 1 - 2 sin^2(a/2) keeps its deviation
        const TS sh = TS(sinf(float(alpha * TS(0.5))));
        ca = TS(1) - TS(2) * sh * sh;
        sa = TS(sinf(float(alpha)));
    } else {
        ca = cos(alpha);
        sa = sin(alpha);
    }
    const TS n2x = nx * ca - tx * sa, n2y = ny * ca - ty * sa;
    const TS P0x = xT[0] * nx, P0y = xT[0] * ny;
    const TS Fx = P0x - n2x / kappa, Fy = P0y - n2y / kappa;
    const TS rx = (P0x - Fx) * fabs(kappa), ry = (P0y - Fy) * fabs(kappa);
    const TS wx = -TS(X[0]) - Fx, wy = -TS(Y[0]) - Fy;
    const TS dist = sqrt_t(wx * wx + wy * wy);
    const TS ex = wx / dist, ey = wy / dist;
    const TS tpx = -sgf * ey, tpy = sgf * ex;
    const TS cot = (xL[1] - xL[0]) / ds0;
    const TS psi = atan2_t<FT>(sgf * (ex * ry - ey * rx), ex * rx + ey * ry);
    const int qf = sgf > TS(0) ? -1 : 1;
    o.pt = double(TS(kKpt * p.bfield) * R);
    o.phi = double(atan2_t<FT>(tpy, tpx));
    o.cot = double(cot);
    o.dxy = double(TS(qf) * (dist - R));
    o.dz = double(xL[0] - cot * (R * psi));
    o.chi2 = double(chi2T + chi2L);
    o.q = (int8_t)qf;
    o.status = 0;
}

__device__ __forceinline__ void fit_dispatch(int n, const float *X, const float *Y,
                                             const float *Z, const uint8_t *L,
                                             const DevParams &p, FitOut &o)
{
    if (p.fit_mode == FIT_MIXED) fit_track<double, double, double, true>(n, X, Y, Z, L, p, o);
    else if (p.fit_mode == FIT_FP32) fit_track<float, float, float, false>(n, X, Y, Z, L, p, o);
    else fit_track<double, double, double, false>(n, X, Y, Z, L, p, o);
}

__global__ void __launch_bounds__(256) k_fit(DevBatch b, DevParams p, uint32_t total)
{
    const uint32_t n_chunks = total / kChunk;
    for (uint32_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint32_t t = ch * kChunk + threadIdx.x;
        const uint32_t e = b.tup_chunk[ch];
        const uint32_t t0 = b.tup_off[e];
        const uint32_t nt = min(b.cnt[C_TUPLES * b.E + e], b.tup_off[e + 1] - t0);
        if (t - t0 >= nt) continue;
        const uint32_t rank = b.tup_rank[t];
        if (rank == kNone) continue;
        const uint32_t o = b.out_evt[e] + rank;
        const int n = b.tup_n[t];
        float X[kMaxHits], Y[kMaxHits], Z[kMaxHits];
        uint8_t L[kMaxHits];
        for (int h = 0; h < kMaxHits; ++h) {
            const uint32_t pos = b.tup_hits[(size_t)t * kMaxHits + h];
            if (h < n) {
                const float4 v = b.hs[pos];
                const uint32_t meta = b.hmeta[pos];
                X[h] = v.x; Y[h] = v.y; Z[h] = v.z;
                L[h] = (uint8_t)(meta >> kLocalBits);
                b.o_hits[(size_t)o * kMaxHits + h] = meta & kLocalMask;
            } else {
                b.o_hits[(size_t)o * kMaxHits + h] = kNone;
            }
        }
        FitOut f;
        fit_dispatch(n, X, Y, Z, L, p, f);
        b.o_nh[o] = (uint8_t)n;
        b.o_pt[o] = f.pt; b.o_phi[o] = f.phi; b.o_cot[o] = f.cot;
        b.o_dxy[o] = f.dxy; b.o_dz[o] = f.dz; b.o_chi2[o] = f.chi2;
        b.o_q[o] = f.q; b.o_status[o] = f.status;
    }
}

void launch_fit(const DevBatch &b, const DevParams &p, uint32_t total, cudaStream_t s, int sms)
{
    uint64_t blocks = total / kChunk;
    uint64_t cap = (uint64_t)sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) return;
    k_fit<<<(unsigned)blocks, kChunk, 0, s>>>(b, p, total);
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
        fit_dispatch(n <= (int)stride ? n : 0, X, Y, Z, L, p, f);
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
