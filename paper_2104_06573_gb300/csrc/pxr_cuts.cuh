// The three cut quantities of the CA seeding (doublet phi window, r-z alignment, transverse DCA).
//
// FP64 form.  Each quantity is a fixed sequence of correctly rounded + - * / sqrt written with
// explicit round-to-nearest intrinsics, so that no multiply-add is fused and the decision equals
// that of any IEEE double implementation evaluating the same sequence.  Inputs are FP32 hit
// coordinates promoted exactly to double.
//
// FP32 form.  The same quantity in float plus a rigorous bound on its distance from the exact real
// value.  If the float margin to the threshold exceeds the bound, the float decision equals the
// exact decision (and the double one, whose own error is ~2^-29 times smaller); otherwise the
// FP64 form decides.  Bounds use u = 2^-24 and the running-error rule
// |fl(expression) - expression| <= gamma_k * (expression evaluated on absolute values).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pxr {

constexpr float kU = 5.9604645e-8f;  // 2^-24

// ------------------------------------------------------------------------------------------
// FP64 forms
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double radius64(double x, double y)
{
    return __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
}

// x_i x_o + y_i y_o >= (cw r_i) r_o
__device__ __forceinline__ bool doublet64(double xi, double yi, double ri, double xo, double yo,
                                          double ro, double cw)
{
    double dot = __dadd_rn(__dmul_rn(xi, xo), __dmul_rn(yi, yo));
    double rhs = __dmul_rn(__dmul_rn(cw, ri), ro);
    return dot >= rhs;
}

// length of an r-z segment: sqrt(dr*dr + dz*dz), dr = r_b - r_a, dz = z_b - z_a
__device__ __forceinline__ double seglen64(double ra, double za, double rb, double zb)
{
    double dr = __dsub_rn(rb, ra), dz = __dsub_rn(zb, za);
    return __dsqrt_rn(__dadd_rn(__dmul_rn(dr, dr), __dmul_rn(dz, dz)));
}

// |a_r b_z - a_z b_r| <= (t |a|) |b|
__device__ __forceinline__ bool theta64(double ri, double zi, double rj, double zj, double rk,
                                        double zk, double na, double nb, double t)
{
    double ar = __dsub_rn(rj, ri), az = __dsub_rn(zj, zi);
    double br = __dsub_rn(rk, rj), bz = __dsub_rn(zk, zj);
    double lhs = fabs(__dsub_rn(__dmul_rn(ar, bz), __dmul_rn(az, br)));
    double rhs = __dmul_rn(__dmul_rn(t, na), nb);
    return lhs <= rhs;
}

// distance of the origin from the circle through p_i, p_j, p_k (see the parameter docs)
__device__ __forceinline__ double dca64(double xi, double yi, double xj, double yj, double xk,
                                        double yk)
{
    double ux = __dsub_rn(xj, xi), uy = __dsub_rn(yj, yi);
    double vx = __dsub_rn(xk, xi), vy = __dsub_rn(yk, yi);
    double D = __dmul_rn(2.0, __dsub_rn(__dmul_rn(ux, vy), __dmul_rn(uy, vx)));
    if (D == 0.0) {
        double cr = __dsub_rn(__dmul_rn(xi, vy), __dmul_rn(yi, vx));
        return __ddiv_rn(fabs(cr), __dsqrt_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy))));
    }
    double uu = __dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy));
    double vv = __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy));
    double cpx = __ddiv_rn(__dsub_rn(__dmul_rn(uu, vy), __dmul_rn(vv, uy)), D);
    double cpy = __ddiv_rn(__dsub_rn(__dmul_rn(vv, ux), __dmul_rn(uu, vx)), D);
    double cx = __dadd_rn(xi, cpx), cy = __dadd_rn(yi, cpy);
    double R = __dsqrt_rn(__dadd_rn(__dmul_rn(cpx, cpx), __dmul_rn(cpy, cpy)));
    double pw = __dsub_rn(__dmul_rn(2.0, __dadd_rn(__dmul_rn(cx, xi), __dmul_rn(cy, yi))),
                          __dadd_rn(__dmul_rn(xi, xi), __dmul_rn(yi, yi)));
    double den = __dadd_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy))), R);
    return __ddiv_rn(fabs(pw), den);
}

// ------------------------------------------------------------------------------------------
// FP32 forms with guard band.  Return 1 pass, 0 fail, -1 undecided (use the FP64 form).
// ------------------------------------------------------------------------------------------

// Doublet.  dot = fma(xi, xo, yi*yo) has error <= 2.01u (|xi xo| + |yi yo|) <= 2.01u ri ro;
// rhs = (cw32 ri32) ro32 with ri32 = fl(ri64) carries 5 relative roundings (cw, ri, ro, two
// products) <= 5.01u ri ro; the difference one more.  8.1u ri ro <= 1e-6 ri32 ro32.
__device__ __forceinline__ int doublet32(float4 hi, float4 ho, float cw32)
{
    float dot = __fmaf_rn(hi.x, ho.x, __fmul_rn(hi.y, ho.y));
    float rr = __fmul_rn(hi.w, ho.w);
    float rhs = __fmul_rn(__fmul_rn(cw32, hi.w), ho.w);
    float d = __fsub_rn(dot, rhs);
    float B = __fmul_rn(1e-6f, rr);
    if (d > B) return 1;
    if (d < -B) return 0;
    return -1;
}

// r-z alignment.  a = (ar, az), b = (br, bz) from float radii (ri32 = fl(ri64), error <= u r)
// and exact float z.  Component errors: |d ar| <= u (ri + rj + |ar|), |d az| <= u |az|; take
// Ea = u (ri + rj + |ar| + |az|) for both (and Eb alike).  Then
//   |cross32 - cross| <= sqrt2 (Ea |b| + Eb |a|) + 3u |a||b|,
//   |rhs32 - rhs|     <= t (sqrt2 (Ea |b| + Eb |a|) + 4u |a||b|) + 3u t |a||b|,
// and the band below doubles their sum (second-order terms and the subtraction included).
struct RZ32 {
    float ar, az, na, Ea;
};

__device__ __forceinline__ RZ32 rz32(float4 ha, float4 hb)
{
    RZ32 s;
    s.ar = __fsub_rn(hb.w, ha.w);
    s.az = __fsub_rn(hb.z, ha.z);
    s.na = __fsqrt_rn(__fmaf_rn(s.ar, s.ar, __fmul_rn(s.az, s.az)));
    s.Ea = kU * (ha.w + hb.w + fabsf(s.ar) + fabsf(s.az));
    return s;
}

__device__ __forceinline__ int theta32(const RZ32 &a, const RZ32 &b, float t32)
{
    float cross = __fmaf_rn(a.ar, b.az, -__fmul_rn(a.az, b.ar));
    float lhs = fabsf(cross);
    float nn = __fmul_rn(a.na, b.na);
    float rhs = __fmul_rn(__fmul_rn(t32, a.na), b.na);
    float d = __fsub_rn(lhs, rhs);
    float B = 2.0f * (1.4143f * (1.0f + t32) * (a.Ea * b.na + b.Ea * a.na) + 8.0f * kU * nn);
    if (d < -B) return 1;
    if (d > B) return 0;
    return -1;
}

// DCA, division-free: with G = |p_i|^2 D + 2 N.p_i and H = |p_i D + N| + |N|
// (N = (|u|^2 v_y - |v|^2 u_y, |v|^2 u_x - |u|^2 v_x)), dca = |G| / H, so dca <= d iff
// |G| <= d H.  Each of G and H is a polynomial of at most 14 rounded operations on inputs with
// relative error u; its error is below gamma_16 times the same polynomial on absolute values
// (Gabs, Habs).  The band takes twice that.  Habs bounds each square root of a sum of two
// squares by the sum of the two absolute values (larger, so the band stays an upper bound).
__device__ __forceinline__ int dca32(float xi, float yi, float xj, float yj, float xk, float yk,
                                     float d)
{
    float ux = __fsub_rn(xj, xi), uy = __fsub_rn(yj, yi);
    float vx = __fsub_rn(xk, xi), vy = __fsub_rn(yk, yi);
    float a1 = __fmul_rn(ux, vy), a2 = __fmul_rn(uy, vx);
    float D = 2.0f * __fsub_rn(a1, a2);
    float Dabs = 2.0f * (fabsf(a1) + fabsf(a2));
    float uu = __fmaf_rn(ux, ux, __fmul_rn(uy, uy));
    float vv = __fmaf_rn(vx, vx, __fmul_rn(vy, vy));
    float Nx = __fsub_rn(__fmul_rn(uu, vy), __fmul_rn(vv, uy));
    float Ny = __fsub_rn(__fmul_rn(vv, ux), __fmul_rn(uu, vx));
    float Nxa = uu * fabsf(vy) + vv * fabsf(uy);
    float Nya = vv * fabsf(ux) + uu * fabsf(vx);
    float pp = __fmaf_rn(xi, xi, __fmul_rn(yi, yi));
    float G = __fmaf_rn(pp, D, 2.0f * __fmaf_rn(Nx, xi, __fmul_rn(Ny, yi)));
    float Gabs = pp * Dabs + 2.0f * (Nxa * fabsf(xi) + Nya * fabsf(yi));
    float qx = __fmaf_rn(xi, D, Nx), qy = __fmaf_rn(yi, D, Ny);
    float H = __fadd_rn(__fsqrt_rn(__fmaf_rn(qx, qx, __fmul_rn(qy, qy))),
                        __fsqrt_rn(__fmaf_rn(Nx, Nx, __fmul_rn(Ny, Ny))));
    float qxa = fabsf(xi) * Dabs + Nxa, qya = fabsf(yi) * Dabs + Nya;
    float Habs = qxa + qya + Nxa + Nya;
    float q = __fsub_rn(fabsf(G), __fmul_rn(d, H));
    float B = 2.0f * 16.0f * kU * (Gabs + d * Habs) * 1.01f;
    if (!(Gabs < 1e30f) || !(Habs < 1e30f)) return -1;
    if (q < -B) return 1;
    if (q > B) return 0;
    return -1;
}

}  // namespace pxr
