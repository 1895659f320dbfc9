/*
 * FP64 CPU oracle of the pixel-track hot path.  TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the CPU-baseline leg of the benchmark are the only callers.  The product path never
 * links, loads or calls this file.  It shares no code, header or table with the CUDA library.
 *
 * What it computes.  The paper (§2, "Patatrack Heterogeneous Pixel Reconstruction") states that the
 * Tracks module "forms n-tuplets from the hits, and fits the hit n-tuplets to obtain track
 * parameters" and gives no further definition.  The steps below follow the published method that
 * sentence refers to, in the reading fixed for this project:
 *
 *   doublets : every (inner, outer) hit pair on an allowed layer pair whose azimuths differ by at
 *              most w, tested as  x_i x_o + y_i y_o >= cos(w) r_i r_o  (no atan2 needed).
 *   CA edges : cell A=(i,j) -> cell B=(j,k) when the r-z segments are aligned,
 *              |a_r b_z - a_z b_r| <= t |a| |b|, and the circle through the three hits passes
 *              within d of the beam line (transverse origin).
 *   ntuplets : depth-first walk from every root cell; a path is emitted when it cannot be
 *              extended or has reached max_hits, and has at least min_hits hits; optionally the
 *              paths that are strict suffixes of other emitted paths are removed.
 *   fit      : broken-line helix fit (V. Blobel, NIM A 566 (2006) 14): a transverse fit of offsets
 *              from a three-point reference circle plus one curvature correction, and a line fit
 *              in (s, z), both with multiple-scattering kinks at the inner hits; normal equations
 *              solved by Cholesky; conversion to (pT, phi, cot theta, dxy, dz) at the point of
 *              closest approach to the beam line.
 *
 * Arithmetic rules.  Inputs are FP32 values promoted exactly to double.  Every cut quantity is a
 * fixed sequence of correctly rounded + - * / sqrt in the order written below; this file must be
 * compiled with -ffp-contract=off so that no multiply-add is fused.  Comparisons are inclusive.
 * cos(w) is an input, computed once by the caller.
 *
 * The oracle is plain and slow on purpose: the doublet search tests every hit pair of every
 * allowed layer pair, and the cell graph is walked recursively.  (A windowed doublet search,
 * equal to the all-pairs one entry by entry, serves the timed CPU baseline.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_LAYERS 16
#define ORC_MAX_PAIRS 32
#define ORC_MAXH 8                    /* hit slots per ntuplet */
#define ORC_K_PT 0.299792458e-2       /* pT [GeV] = K B[T] R[cm] */
#define ORC_TWO_PI 6.283185307179586476925286766559

typedef struct {
    uint32_t n_layers;
    uint8_t layer_is_disk[ORC_MAX_LAYERS];
    uint32_t n_pairs;
    uint8_t pair_inner[ORC_MAX_PAIRS];
    uint8_t pair_outer[ORC_MAX_PAIRS];
    uint32_t root_mask;
    uint32_t drop_suffixes;
    uint32_t min_hits;
    uint32_t max_hits;
    double cos_phi_window;
    double theta_cut;
    double dca_cut;
    double bfield;
    double sigma_rphi;
    double sigma_z;
    double x_over_x0;
} orc_params;

typedef struct {
    double pt, phi, cot_theta, dxy, dz, chi2;
    int32_t charge;
    int32_t status;   /* 0 ok, 1 collinear prefit, 2 zero curvature, 3 Cholesky, 4 bad MS input */
} orc_track;

typedef struct {
    uint32_t n_hits;
    uint32_t n_cells;
    uint32_t *cell_in, *cell_out;         /* caller hit indices */
    uint32_t n_edges;
    uint32_t *edge_a, *edge_b;            /* cell indices */
    uint32_t n_tuples;
    uint8_t *tup_n;
    uint32_t *tup_hits;                   /* [n_tuples * ORC_MAXH], unused slots 0xFFFFFFFF */
    orc_track *fit;
} orc_result;

/* ------------------------------------------------------------------------------------------ */
/* Cut quantities (reading of the CA cuts: doublet window, r-z alignment, transverse DCA)      */
/* ------------------------------------------------------------------------------------------ */

double orc_radius(double x, double y) { return sqrt(x * x + y * y); }

/* Doublet cut: |delta phi| <= w  <=>  x_i x_o + y_i y_o >= cos(w) r_i r_o. */
int orc_doublet_pass(double xi, double yi, double xo, double yo, double cw)
{
    double ri = orc_radius(xi, yi);
    double ro = orc_radius(xo, yo);
    double dot = xi * xo + yi * yo;
    double rhs = cw * ri * ro;
    return dot >= rhs;
}

/* r-z alignment: a = (r_j - r_i, z_j - z_i), b = (r_k - r_j, z_k - z_j),
 * pass iff |a_r b_z - a_z b_r| <= t |a| |b|  (|sin| of the bend angle at hit j). */
int orc_theta_pass(double ri, double zi, double rj, double zj, double rk, double zk, double t)
{
    double ar = rj - ri, az = zj - zi;
    double br = rk - rj, bz = zk - zj;
    double na = sqrt(ar * ar + az * az);
    double nb = sqrt(br * br + bz * bz);
    double lhs = fabs(ar * bz - az * br);
    double rhs = t * na * nb;
    return lhs <= rhs;
}

/* Distance of the transverse origin from the circle through p_i, p_j, p_k.
 * u = p_j - p_i, v = p_k - p_i, D = 2 (u x v); centre offset c' = ((|u|^2 v_y - |v|^2 u_y) / D,
 * (|v|^2 u_x - |u|^2 v_x) / D); c = p_i + c', R = |c'|; since |c|^2 - R^2 = 2 c.p_i - |p_i|^2,
 * dca = |2 c.p_i - |p_i|^2| / (|c| + R).  For D == 0 the three points are collinear and the
 * distance to the line through p_i and p_k is returned. */
double orc_dca(double xi, double yi, double xj, double yj, double xk, double yk)
{
    double ux = xj - xi, uy = yj - yi;
    double vx = xk - xi, vy = yk - yi;
    double D = 2.0 * (ux * vy - uy * vx);
    if (D == 0.0) {
        double cr = xi * vy - yi * vx;
        return fabs(cr) / sqrt(vx * vx + vy * vy);
    }
    double uu = ux * ux + uy * uy;
    double vv = vx * vx + vy * vy;
    double cpx = (uu * vy - vv * uy) / D;
    double cpy = (vv * ux - uu * vx) / D;
    double cx = xi + cpx, cy = yi + cpy;
    double R = sqrt(cpx * cpx + cpy * cpy);
    double pw = 2.0 * (cx * xi + cy * yi) - (xi * xi + yi * yi);
    return fabs(pw) / (sqrt(cx * cx + cy * cy) + R);
}

int orc_dca_pass(double xi, double yi, double xj, double yj, double xk, double yk, double d)
{
    return orc_dca(xi, yi, xj, yj, xk, yk) <= d;
}

/* ------------------------------------------------------------------------------------------ */
/* Growable arrays                                                                             */
/* ------------------------------------------------------------------------------------------ */
typedef struct { uint32_t *a; size_t n, cap; } u32vec;

static int push(u32vec *v, uint32_t x)
{
    if (v->n == v->cap) {
        size_t nc = v->cap ? 2 * v->cap : 1024;
        uint32_t *p = (uint32_t *)realloc(v->a, nc * sizeof(uint32_t));
        if (!p) return -1;
        v->a = p;
        v->cap = nc;
    }
    v->a[v->n++] = x;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Broken-line normal equations (shared by the transverse and the line fit)                    */
/* ------------------------------------------------------------------------------------------ */
#define ORC_MAXM (ORC_MAXH + 1)

/* Dense Cholesky A = L L^T without pivoting, then forward and back substitution. */
static int chol_solve(int m, const double *A, const double *b, double *x)
{
    double L[ORC_MAXM * ORC_MAXM];
    double y[ORC_MAXM];
    memset(L, 0, sizeof(L));
    for (int j = 0; j < m; ++j) {
        double s = A[j * m + j];
        for (int k = 0; k < j; ++k) s -= L[j * m + k] * L[j * m + k];
        if (!(s > 0.0)) return -1;
        L[j * m + j] = sqrt(s);
        for (int i = j + 1; i < m; ++i) {
            double t = A[i * m + j];
            for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
            L[i * m + j] = t / L[j * m + j];
        }
    }
    for (int i = 0; i < m; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= L[i * m + k] * y[k];
        y[i] = t / L[i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < m; ++k) t -= L[k * m + i] * x[k];
        x[i] = t / L[i * m + i];
    }
    return 0;
}

/*
 * Broken line over n points at path lengths s[0..n-1] with measurements meas[i] of weight w[i].
 * Unknowns: offsets x[0..n-1] and, when curv != 0, one curvature correction x[n].
 * Kink at each inner point j = 1..n-2:
 *     beta_j = (x[j+1]-x[j])/ds_j - (x[j]-x[j-1])/ds_{j-1} + curv * (ds_{j-1}+ds_j)/2 * x[n]
 * with variance kvar[j].  The curvature term is written with a plus sign because an increase of
 * the curvature magnitude pulls the path towards the centre, i.e. the outward offset has second
 * derivative -x[n].  The result is the minimiser of
 *     chi2 = sum w (meas - x)^2 + sum beta^2 / kvar.
 *
 * The minimiser is computed in the parameters theta = (x[0], slope of the first segment,
 * [x[n]], beta_1 .. beta_{n-2}), which describe the same paths one to one: the slope of segment
 * m is slope_0 + sum_{j=1..m} (beta_j - curv (ds_{j-1}+ds_j)/2 x[n]), so
 *     x[i] = x[0] + slope_0 (s_i - s_0) + sum_{1<=j<i} (beta_j - curv c_j x[n]) (s_i - s_j),
 *     c_j = (s_{j+1} - s_{j-1}) / 2,
 * and chi2 = |W^(1/2) (meas - J theta)|^2 + sum beta_j^2 / kvar_j.  Its normal matrix
 * J^T W J + diag(0, .., 1/kvar_j) keeps the kink weights on the diagonal: with little material
 * they reach 1e20 next to measurement weights of 1e6, and the normal equations written in the
 * offsets x would mix the two in every entry, where their FP64 rounding leaves the straight-line
 * part of the solution with errors of 1e-3; here they stay apart and the solve keeps FP64
 * accuracy.  Dense Cholesky; x = J theta.  Ainv (optional) receives the inverse normal matrix in
 * the offsets (x[0..n-1], x[n]): T N^-1 T^T with T the map from theta to them.
 * Returns 0 on success and stores the minimum in *chi2.
 */
static int bl_solve(int n, const double *s, const double *meas, const double *w,
                    const double *kvar, int curv, double *x, double *chi2, double *Ainv)
{
    const int g = curv ? 3 : 2;                 /* x[0], slope_0, [curvature correction] */
    const int m = n + (curv ? 1 : 0);           /* = g + (n - 2) */
    double J[ORC_MAXH][ORC_MAXM];               /* d x_i / d theta_k */
    double N[ORC_MAXM * ORC_MAXM], b[ORC_MAXM], th[ORC_MAXM];
    if (n < 2 || n > ORC_MAXH) return -1;
    memset(J, 0, sizeof(J));
    for (int i = 0; i < n; ++i) {
        J[i][0] = 1.0;
        J[i][1] = s[i] - s[0];
        for (int j = 1; j < i && j + 1 < n; ++j) {
            J[i][g + j - 1] = s[i] - s[j];
            if (curv) J[i][2] -= 0.5 * (s[j + 1] - s[j - 1]) * (s[i] - s[j]);
        }
    }
    for (int r = 0; r < m; ++r) {
        b[r] = 0.0;
        for (int i = 0; i < n; ++i) b[r] += J[i][r] * w[i] * meas[i];
        for (int c = 0; c < m; ++c) {
            double a = 0.0;
            for (int i = 0; i < n; ++i) a += J[i][r] * w[i] * J[i][c];
            N[r * m + c] = a;
        }
    }
    for (int j = 1; j + 1 < n; ++j) N[(g + j - 1) * m + (g + j - 1)] += 1.0 / kvar[j];
    if (chol_solve(m, N, b, th) != 0) return -1;
    for (int i = 0; i < n; ++i) {
        double v = 0.0;
        for (int k = 0; k < m; ++k) v += J[i][k] * th[k];
        x[i] = v;
    }
    if (curv) x[n] = th[2];
    /* inverse normal matrix in the offsets: T N^-1 T^T, T's rows the J rows and, for the
     * curvature correction, the unit row of theta_2 */
    if (Ainv) {
        double Ninv[ORC_MAXM * ORC_MAXM], T[ORC_MAXM][ORC_MAXM];
        for (int k = 0; k < m; ++k) {
            double e[ORC_MAXM], col[ORC_MAXM];
            memset(e, 0, sizeof(e));
            e[k] = 1.0;
            if (chol_solve(m, N, e, col) != 0) return -1;
            for (int r = 0; r < m; ++r) Ninv[r * m + k] = col[r];
        }
        memset(T, 0, sizeof(T));
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < m; ++k) T[i][k] = J[i][k];
        if (curv) T[n][2] = 1.0;
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c) {
                double a = 0.0;
                for (int k = 0; k < m; ++k)
                    for (int l = 0; l < m; ++l) a += T[r][k] * Ninv[k * m + l] * T[c][l];
                Ainv[r * m + c] = a;
            }
    }
    double c2 = 0.0;
    for (int i = 0; i < n; ++i) c2 += w[i] * (meas[i] - x[i]) * (meas[i] - x[i]);
    for (int j = 1; j + 1 < n; ++j) c2 += th[g + j - 1] * th[g + j - 1] / kvar[j];
    *chi2 = c2;
    return 0;
}

int orc_bl_solve(int n, const double *s, const double *meas, const double *w, const double *kvar,
                 int curv, double *x, double *chi2)
{
    return bl_solve(n, s, meas, w, kvar, curv, x, chi2, NULL);
}

/* ------------------------------------------------------------------------------------------ */
/* Broken-line helix fit of one ntuplet                                                        */
/* ------------------------------------------------------------------------------------------ */
/*
 * Steps (reading of "fits the hit n-tuplets to obtain track parameters", §2):
 *  1. local frame at hit 0; reference circle through hits 0, n/2, n-1 (centre C, radius R0);
 *     orientation sgn = sign(D) (+1 counter-clockwise), charge q = -sgn (B along +z).
 *  2. path length s_i = R0 * (signed angle from hit 0 to hit i about C, along the motion);
 *     transverse residual y_i = |p_i - C| - R0 (outward positive), evaluated as
 *     (|p_i|^2 - 2 p_i.C) / (|p_i - C| + R0) to avoid cancellation at large R0.
 *  3. multiple scattering at inner hits: Highland angle theta0 = 0.0136/p sqrt(x) (1 + 0.038 ln x)
 *     with p = pT0 sqrt(1 + cot^2), pT0 = K B R0, cot from hits 0 and n-1 in (s, z), and the
 *     traversed thickness x = x_over_x0 * sqrt(1+cot^2) on barrel layers, x_over_x0 *
 *     sqrt(1+cot^2)/|cot| on disks.  Kink variances: transverse theta0^2 (1+cot^2) (a deflection
 *     theta0 perpendicular to the track changes the transverse direction by theta0 / sin(theta)),
 *     line theta0^2 (1+cot^2)^2 (d cot = -d theta / sin^2 theta).
 *  4. transverse broken line with curvature correction (weights 1/sigma_rphi^2).
 *  5. line broken line in (s, z) (weights 1/sigma_z^2 on barrel layers; on disks, where z is fixed
 *     and the radius is measured with sigma_z, the z-equivalent error sigma_z |cot|).
 *  6. conversion: curvature kappa = 1/R0 + delta (relative to the bending sense of the reference
 *     circle; a negative kappa bends the other way and flips the charge); fitted point at hit 0 =
 *     hit 0 + u_0 along the outward normal; direction rotated towards the outward normal by
 *     u'(0) = (u_1-u_0)/ds_0 + delta ds_0/2; fitted centre = that point - (rotated normal)/kappa;
 *     point of closest approach (PCA) to the transverse origin;
 *     dxy = q (|C_fit - O| - R)  (positive for q > 0 when the origin lies outside the circle);
 *     phi = direction of motion at the PCA; pT = K B R; cot = (v_1 - v_0)/ds_0;
 *     dz = v_0 - cot * (arc length from the PCA to hit 0).
 */
/* Step 6 as a function of the fitted values q = (u_0, u_1, delta, v_0, v_1) and the reference
 * circle's geometry (also evaluated around q for the covariance's Jacobian). */
typedef struct {
    double R0, Cx, Cy, sgn, x0, y0, ds0, kB;
} conv_geom;

static int bl_convert(const conv_geom *G, const double *q, orc_track *out)
{
    double delta = q[2];
    double kappa = 1.0 / G->R0 + delta;               /* > 0: bends like the reference circle */
    if (kappa == 0.0 || !isfinite(kappa)) return 2;
    double R = 1.0 / fabs(kappa);
    double sgn = G->sgn;
    double sgf = kappa > 0.0 ? sgn : -sgn;            /* orientation about the fitted centre */
    int qf = sgf > 0.0 ? -1 : 1;
    double ds0 = G->ds0;
    double alpha = (q[1] - q[0]) / ds0 + 0.5 * delta * ds0;
    double nx = -G->Cx / G->R0, ny = -G->Cy / G->R0;  /* outward normal at hit 0 */
    double tx = -sgn * ny, ty = sgn * nx;             /* direction of motion at hit 0 */
    double ca = cos(alpha), sa = sin(alpha);
    double n2x = nx * ca - tx * sa, n2y = ny * ca - ty * sa;
    double P0x = q[0] * nx, P0y = q[0] * ny;
    double Fx = P0x - n2x / kappa, Fy = P0y - n2y / kappa;   /* fitted centre */
    double rx = (P0x - Fx) * fabs(kappa), ry = (P0y - Fy) * fabs(kappa); /* centre -> hit 0 */
    double wx = -G->x0 - Fx, wy = -G->y0 - Fy;        /* centre -> transverse origin */
    double dist = sqrt(wx * wx + wy * wy);
    double ex = wx / dist, ey = wy / dist;
    double tpx = -sgf * ey, tpy = sgf * ex;           /* direction of motion at the PCA */
    double cot = (q[4] - q[3]) / ds0;
    double psi = atan2(sgf * (ex * ry - ey * rx), ex * rx + ey * ry);
    out->pt = G->kB * R;
    out->phi = atan2(tpy, tpx);
    out->cot_theta = cot;
    out->dxy = qf * (dist - R);
    out->dz = q[3] - cot * (R * psi);
    out->charge = qf;
    out->status = 0;
    return 0;
}

/* The five parameters of the covariance: q/pT (charge over pT, 1/GeV), phi, cot, dxy, dz. */
static void cov_params(const orc_track *t, double *v)
{
    v[0] = t->charge / t->pt;
    v[1] = t->phi;
    v[2] = t->cot_theta;
    v[3] = t->dxy;
    v[4] = t->dz;
}

/*
 * Covariance of (q/pT, phi, cot, dxy, dz): the fitted values q have the covariance of the
 * linear least-squares problems, the inverse normal matrices (u_0, u_1, delta from the
 * transverse fit, v_0, v_1 from the line fit; the two fits are independent); the conversion is
 * linearised around q by a five-point central difference in each q_k with step 1e-3 of its
 * standard deviation.  cov15 receives the upper triangle row by row.
 */
static int bl_cov(const conv_geom *G, const double *q, const double *AT, int mT, int n,
                  const double *AL, double *cov15)
{
    double C[5][5];
    memset(C, 0, sizeof(C));
    const int it[3] = {0, 1, n};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) C[a][b] = AT[it[a] * mT + it[b]];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) C[3 + a][3 + b] = AL[a * n + b];
    double J[5][5];
    for (int k = 0; k < 5; ++k) {
        if (!(C[k][k] > 0.0)) return -1;
        const double h = 1e-3 * sqrt(C[k][k]);
        double v[4][5];
        const double off[4] = {-2.0, -1.0, 1.0, 2.0};
        for (int t = 0; t < 4; ++t) {
            double qq[5];
            orc_track tr;
            for (int i = 0; i < 5; ++i) qq[i] = q[i];
            qq[k] += off[t] * h;
            if (bl_convert(G, qq, &tr) != 0) return -1;
            cov_params(&tr, v[t]);
        }
        for (int i = 0; i < 5; ++i) {
            double d1 = v[2][i] - v[1][i], d2 = v[3][i] - v[0][i];
            if (i == 1) {                               /* azimuth differences modulo 2 pi */
                d1 = remainder(d1, ORC_TWO_PI);
                d2 = remainder(d2, ORC_TWO_PI);
            }
            J[i][k] = (8.0 * d1 - d2) / (12.0 * h);
        }
    }
    int o = 0;
    for (int i = 0; i < 5; ++i)
        for (int j = i; j < 5; ++j) {
            double acc = 0.0;
            for (int a = 0; a < 5; ++a)
                for (int b = 0; b < 5; ++b) acc += J[i][a] * C[a][b] * J[j][b];
            cov15[o++] = acc;
        }
    return 0;
}

static int fit_core(int n, const double *X, const double *Y, const double *Z, const uint16_t *lay,
                    const orc_params *P, orc_track *out, double *cov15)
{
    double px[ORC_MAXH], py[ORC_MAXH], s[ORC_MAXH], yres[ORC_MAXH];
    double wT[ORC_MAXH], wL[ORC_MAXH], kvT[ORC_MAXH], kvL[ORC_MAXH];
    double xT[ORC_MAXM], xL[ORC_MAXM];
    double chi2T = 0.0, chi2L = 0.0;
    memset(out, 0, sizeof(*out));
    if (n < 3 || n > ORC_MAXH) { out->status = 4; return -1; }

    /* 1. local frame and reference circle */
    double x0 = X[0], y0 = Y[0];
    for (int i = 0; i < n; ++i) { px[i] = X[i] - x0; py[i] = Y[i] - y0; }
    int b = n / 2, c = n - 1;
    double ux = px[b], uy = py[b], vx = px[c], vy = py[c];
    double D = 2.0 * (ux * vy - uy * vx);
    if (D == 0.0) { out->status = 1; return -1; }
    double uu = ux * ux + uy * uy, vv = vx * vx + vy * vy;
    double Cx = (uu * vy - vv * uy) / D;
    double Cy = (vv * ux - uu * vx) / D;
    double R0 = sqrt(Cx * Cx + Cy * Cy);
    double sgn = D > 0.0 ? 1.0 : -1.0;

    /* 2. path lengths and residuals */
    double ax = -Cx, ay = -Cy;
    for (int i = 0; i < n; ++i) {
        double dx = px[i] - Cx, dy = py[i] - Cy;
        /* |p - C| - R0 written without cancellation: the circle passes through the local origin,
         * so |p - C|^2 - R0^2 = |p|^2 - 2 p.C exactly. */
        double pw = (px[i] * px[i] + py[i] * py[i]) - 2.0 * (px[i] * Cx + py[i] * Cy);
        yres[i] = pw / (sqrt(dx * dx + dy * dy) + R0);
        double cr = ax * dy - ay * dx;
        double dt = ax * dx + ay * dy;
        s[i] = R0 * atan2(sgn * cr, dt);
    }

    /* 3. multiple scattering */
    double cot0 = (Z[c] - Z[0]) / (s[c] - s[0]);
    double sec2 = 1.0 + cot0 * cot0;
    double pt0 = ORC_K_PT * P->bfield * R0;
    double p = pt0 * sqrt(sec2);
    for (int i = 0; i < n; ++i) { kvT[i] = 1.0; kvL[i] = 1.0; }
    for (int j = 1; j + 1 < n; ++j) {
        int disk = P->layer_is_disk[lay[j]];
        double path = disk ? sqrt(sec2) / fabs(cot0) : sqrt(sec2);
        double xx = P->x_over_x0 * path;
        double th0 = (0.0136 / p) * sqrt(xx) * (1.0 + 0.038 * log(xx));
        double th2 = th0 * th0;
        kvT[j] = th2 * sec2;
        kvL[j] = th2 * sec2 * sec2;
        if (!(kvT[j] > 0.0) || !(kvL[j] > 0.0)) { out->status = 4; return -1; }
    }
    for (int i = 0; i < n; ++i) {
        wT[i] = 1.0 / (P->sigma_rphi * P->sigma_rphi);
        if (P->layer_is_disk[lay[i]]) {
            double sz = P->sigma_z * fabs(cot0);
            wL[i] = 1.0 / (sz * sz);
        } else {
            wL[i] = 1.0 / (P->sigma_z * P->sigma_z);
        }
    }

    /* 4-5. the two broken lines (and, for the covariance, their inverse normal matrices) */
    double AT[ORC_MAXM * ORC_MAXM], AL[ORC_MAXM * ORC_MAXM];
    if (bl_solve(n, s, yres, wT, kvT, 1, xT, &chi2T, cov15 ? AT : NULL) != 0) { out->status = 3; return -1; }
    if (bl_solve(n, s, Z, wL, kvL, 0, xL, &chi2L, cov15 ? AL : NULL) != 0) { out->status = 3; return -1; }

    /* 6. conversion */
    conv_geom G = {R0, Cx, Cy, sgn, x0, y0, s[1] - s[0], ORC_K_PT * P->bfield};
    const double q[5] = {xT[0], xT[1], xT[n], xL[0], xL[1]};
    int st = bl_convert(&G, q, out);
    if (st) { out->status = st; return -1; }
    out->chi2 = chi2T + chi2L;
    if (cov15 && bl_cov(&G, q, AT, n + 1, n, AL, cov15) != 0) { out->status = 5; return -1; }
    return 0;
}

int orc_fit_one(int n, const double *X, const double *Y, const double *Z, const uint16_t *lay,
                const orc_params *P, orc_track *out)
{
    return fit_core(n, X, Y, Z, lay, P, out, NULL);
}

/* The fit and the covariance of (q/pT, phi, cot, dxy, dz) (15 doubles, upper triangle). */
int orc_fit_cov(int n, const double *X, const double *Y, const double *Z, const uint16_t *lay,
                const orc_params *P, orc_track *out, double *cov15)
{
    return fit_core(n, X, Y, Z, lay, P, out, cov15);
}

/* Fit m ntuplets given as padded rows of ORC_MAXH hits (FP64 coordinates). */
void orc_fit_batch(uint32_t m, const uint8_t *nh, const double *X, const double *Y, const double *Z,
                   const uint16_t *lay, uint32_t stride, const orc_params *P, orc_track *out)
{
    for (uint32_t t = 0; t < m; ++t)
        orc_fit_one(nh[t], X + (size_t)t * stride, Y + (size_t)t * stride, Z + (size_t)t * stride,
                    lay + (size_t)t * stride, P, &out[t]);
}

/* ------------------------------------------------------------------------------------------ */
/* Riemann fit of one ntuplet                                                                  */
/* ------------------------------------------------------------------------------------------ */
/* Eigen-decomposition of a symmetric 3 x 3 matrix by cyclic Jacobi rotations (the textbook
 * method: each rotation zeroes one off-diagonal element; sweeps until they vanish).  On return
 * the diagonal of a holds the eigenvalues and the columns of v the eigenvectors. */
static void jacobi3(double a[3][3], double v[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) v[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        double diag = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
        if (off <= 1e-300 || off <= 1e-18 * diag) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                /* rotation angle that zeroes a[p][q]: tan(2 phi) = 2 a_pq / (a_qq - a_pp) */
                double th = 0.5 * (a[q][q] - a[p][p]) / a[p][q];
                double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 3; ++k) {            /* a <- a J */
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - sn * akq;
                    a[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {            /* a <- J^T a */
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - sn * aqk;
                    a[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {            /* v <- v J */
                    double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - sn * vkq;
                    v[k][q] = sn * vkp + c * vkq;
                }
            }
    }
}

/*
 * Riemann fit (reading of the circle fit on the Riemann paraboloid: Strandlie et al., Comput.
 * Phys. Commun. 131 (2000) 95, in its fast plane-fit form):
 *  1. map each hit (x, y) to (x, y, x^2 + y^2) in the transverse frame of the beam line; fit a
 *     plane c + n.p = 0 (|n| = 1) minimising sum w_i (c + n.p_i)^2 with w_i = 1/sigma_rphi^2:
 *     n is the eigenvector of the smallest eigenvalue of the weighted scatter matrix about the
 *     weighted centroid, c = -n.centroid; the plane cuts the paraboloid in the circle with
 *     centre (-n_x, -n_y) / (2 n_w) and radius^2 = (n_x^2 + n_y^2 - 4 c n_w) / (4 n_w^2);
 *  2. orientation from the turn of hit n-1 relative to hit 0 about the centre (charge = -sgn);
 *     arc lengths s_i from hit 0 along the motion; weighted straight line z = z_0 + cot s
 *     (weights 1/sigma_z^2, disks 1/(sigma_z cot0)^2 as in the broken line);
 *  3. point of closest approach of the circle to the beam line; dxy = q (|C| - R); phi the
 *     direction of motion there; dz = z_0 + cot s_PCA; pT = K B R;
 *     chi2 = sum ((|p_i - C| - R) / sigma_rphi)^2 + sum ((z_i - z_0 - cot s_i) / sigma_z,i)^2.
 * No multiple scattering enters (the fast form).
 */
int orc_riemann_one(int n, const double *X, const double *Y, const double *Z, const uint16_t *lay,
                    const orc_params *P, orc_track *out)
{
    memset(out, 0, sizeof(*out));
    if (n < 3 || n > ORC_MAXH) { out->status = 4; return -1; }
    double w = 1.0 / (P->sigma_rphi * P->sigma_rphi);
    double sw = 0.0, m[3] = {0.0, 0.0, 0.0};
    double pts[ORC_MAXH][3];
    for (int i = 0; i < n; ++i) {
        pts[i][0] = X[i];
        pts[i][1] = Y[i];
        pts[i][2] = X[i] * X[i] + Y[i] * Y[i];
        for (int k = 0; k < 3; ++k) m[k] += w * pts[i][k];
        sw += w;
    }
    for (int k = 0; k < 3; ++k) m[k] /= sw;
    double A[3][3] = {{0}}, V[3][3];
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) A[a][b] += w * (pts[i][a] - m[a]) * (pts[i][b] - m[b]);
    jacobi3(A, V);
    int kmin = 0;
    for (int k = 1; k < 3; ++k)
        if (A[k][k] < A[kmin][kmin]) kmin = k;
    double nx = V[0][kmin], ny = V[1][kmin], nw = V[2][kmin];
    double c = -(nx * m[0] + ny * m[1] + nw * m[2]);
    if (nw == 0.0) { out->status = 1; return -1; }
    double Cx = -nx / (2.0 * nw), Cy = -ny / (2.0 * nw);
    double R2 = (nx * nx + ny * ny - 4.0 * c * nw) / (4.0 * nw * nw);
    if (!(R2 > 0.0) || !isfinite(R2)) { out->status = 2; return -1; }
    double R = sqrt(R2);
    /* orientation: the turn from hit 0 to hit n-1 about the centre */
    double ax = X[0] - Cx, ay = Y[0] - Cy;
    double bx = X[n - 1] - Cx, by = Y[n - 1] - Cy;
    double sgn = (ax * by - ay * bx) > 0.0 ? 1.0 : -1.0;
    int q = sgn > 0.0 ? -1 : 1;
    double s[ORC_MAXH];
    for (int i = 0; i < n; ++i) {
        double dx = X[i] - Cx, dy = Y[i] - Cy;
        s[i] = R * atan2(sgn * (ax * dy - ay * dx), ax * dx + ay * dy);
    }
    /* line */
    double cot0 = (Z[n - 1] - Z[0]) / (s[n - 1] - s[0]);
    double S0 = 0.0, S1 = 0.0, S2 = 0.0, T0 = 0.0, T1 = 0.0, wz[ORC_MAXH];
    for (int i = 0; i < n; ++i) {
        double sz = P->layer_is_disk[lay[i]] ? P->sigma_z * fabs(cot0) : P->sigma_z;
        wz[i] = 1.0 / (sz * sz);
        S0 += wz[i];
        S1 += wz[i] * s[i];
        S2 += wz[i] * s[i] * s[i];
        T0 += wz[i] * Z[i];
        T1 += wz[i] * s[i] * Z[i];
    }
    double det = S0 * S2 - S1 * S1;
    if (!(det > 0.0)) { out->status = 3; return -1; }
    double cot = (S0 * T1 - S1 * T0) / det;
    double z0 = (S2 * T0 - S1 * T1) / det;
    /* point of closest approach to the beam line */
    double dC = sqrt(Cx * Cx + Cy * Cy);
    double ux = -Cx / dC, uy = -Cy / dC;            /* from the centre towards the beam line */
    double Px = Cx + R * ux, Py = Cy + R * uy;
    double tpx = -sgn * (Py - Cy) / R, tpy = sgn * (Px - Cx) / R;
    double s_pca = R * atan2(sgn * (ax * (Py - Cy) - ay * (Px - Cx)), ax * (Px - Cx) + ay * (Py - Cy));
    double chi2 = 0.0;
    for (int i = 0; i < n; ++i) {
        double d = sqrt((X[i] - Cx) * (X[i] - Cx) + (Y[i] - Cy) * (Y[i] - Cy)) - R;
        double e = Z[i] - z0 - cot * s[i];
        chi2 += w * d * d + wz[i] * e * e;
    }
    out->pt = ORC_K_PT * P->bfield * R;
    out->phi = atan2(tpy, tpx);
    out->cot_theta = cot;
    out->dxy = q * (dC - R);
    out->dz = z0 + cot * s_pca;
    out->chi2 = chi2;
    out->charge = q;
    out->status = 0;
    return 0;
}

void orc_riemann_batch(uint32_t m, const uint8_t *nh, const double *X, const double *Y,
                       const double *Z, const uint16_t *lay, uint32_t stride, const orc_params *P,
                       orc_track *out)
{
    for (uint32_t t = 0; t < m; ++t)
        orc_riemann_one(nh[t], X + (size_t)t * stride, Y + (size_t)t * stride,
                        Z + (size_t)t * stride, lay + (size_t)t * stride, P, &out[t]);
}

/* ------------------------------------------------------------------------------------------ */
/* Event reconstruction: doublets -> CA edges -> ntuplets -> fits                              */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    const orc_params *P;
    const uint32_t *cell_in, *cell_out;
    const uint32_t *nbr_first, *nbr;      /* out-edges of each cell */
    const uint16_t *layer;
    u32vec tup;                            /* flat ORC_MAXH-slot rows */
    u32vec tup_n;
    int fail;
} dfs_ctx;

static void emit(dfs_ctx *d, const uint32_t *path_cells, int ncells)
{
    uint32_t row[ORC_MAXH];
    int nh = ncells + 1;
    for (int i = 0; i < ORC_MAXH; ++i) row[i] = 0xFFFFFFFFu;
    row[0] = d->cell_in[path_cells[0]];
    for (int i = 0; i < ncells; ++i) row[i + 1] = d->cell_out[path_cells[i]];
    for (int i = 0; i < ORC_MAXH; ++i)
        if (push(&d->tup, row[i])) d->fail = 1;
    if (push(&d->tup_n, (uint32_t)nh)) d->fail = 1;
}

/* Recursive walk; path holds ncells cells (ncells + 1 hits). */
static void walk(dfs_ctx *d, uint32_t *path, int ncells)
{
    uint32_t last = path[ncells - 1];
    int nh = ncells + 1;
    uint32_t b = d->nbr_first[last], e = d->nbr_first[last + 1];
    if ((uint32_t)nh >= d->P->max_hits || b == e) {
        if ((uint32_t)nh >= d->P->min_hits) emit(d, path, ncells);
        return;
    }
    for (uint32_t k = b; k < e; ++k) {
        path[ncells] = d->nbr[k];
        walk(d, path, ncells + 1);
    }
}

static int row_cmp(const uint32_t *a, const uint32_t *b)
{
    for (int i = 0; i < ORC_MAXH; ++i) {
        if (a[i] < b[i]) return -1;
        if (a[i] > b[i]) return 1;
    }
    return 0;
}

static const uint32_t *g_rows;  /* qsort context (single-threaded use per call) */
static int idx_cmp(const void *pa, const void *pb)
{
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    return row_cmp(g_rows + (size_t)a * ORC_MAXH, g_rows + (size_t)b * ORC_MAXH);
}

void orc_free(orc_result *r)
{
    if (!r) return;
    free(r->cell_in); free(r->cell_out); free(r->edge_a); free(r->edge_b);
    free(r->tup_n); free(r->tup_hits); free(r->fit);
    free(r);
}

/* Doublets by a windowed search (for the timed CPU baseline; the reference definition is the
 * all-pairs search in orc_reconstruct): per layer pair, the outer layer's hits sorted by azimuth;
 * for each inner hit the outer hits whose azimuth lies within phi_window of its own (a binary
 * search at each end, the window wrapping at +-pi, widened by 1e-9 rad, far above the rounding of
 * atan2 and of the cut) are tested with the same cut.  An inner hit's cells are emitted in
 * increasing outer index, so the cell list equals the all-pairs list entry by entry. */
typedef struct { double phi; uint32_t h; } orc_az;

static int az_cmp(const void *pa, const void *pb)
{
    const orc_az *a = (const orc_az *)pa, *b = (const orc_az *)pb;
    return a->phi < b->phi ? -1 : a->phi > b->phi ? 1 : (a->h < b->h ? -1 : a->h > b->h);
}

static int u32_cmp(const void *pa, const void *pb)
{
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    return a < b ? -1 : a > b;
}

/* first index of az[0..m) with phi >= v */
static uint32_t az_lower(const orc_az *az, uint32_t m, double v)
{
    uint32_t lo = 0, hi = m;
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (az[mid].phi < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int doublets_windowed(uint32_t n, const double *x, const double *y, const uint16_t *layer,
                             const orc_params *P, u32vec *ci, u32vec *co)
{
    const double pi = ORC_TWO_PI / 2.0;
    const double W = acos(P->cos_phi_window) + 1e-9;
    orc_az *az = (orc_az *)malloc((n + 1) * sizeof(orc_az));
    uint32_t *cand = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    int rc = -1;
    if (!az || !cand) goto out;
    for (uint32_t p = 0; p < P->n_pairs; ++p) {
        uint32_t Li = P->pair_inner[p], Lo = P->pair_outer[p], m = 0;
        for (uint32_t o = 0; o < n; ++o)
            if (layer[o] == Lo) { az[m].phi = atan2(y[o], x[o]); az[m].h = o; ++m; }
        qsort(az, m, sizeof(orc_az), az_cmp);
        for (uint32_t i = 0; i < n; ++i) {
            if (layer[i] != Li) continue;
            const double phi = atan2(y[i], x[i]);
            double a = phi - W, b = phi + W;
            uint32_t nc = 0;
            /* one or two ranges of azimuth [a, b] (modulo 2 pi) */
            double ra[2][2] = {{a, b}, {1.0, 0.0}};
            if (a < -pi) { ra[0][0] = a + ORC_TWO_PI; ra[0][1] = pi; ra[1][0] = -pi; ra[1][1] = b; }
            else if (b > pi) { ra[0][0] = a; ra[0][1] = pi; ra[1][0] = -pi; ra[1][1] = b - ORC_TWO_PI; }
            if (b - a >= ORC_TWO_PI) { ra[0][0] = -pi - 1.0; ra[0][1] = pi + 1.0; ra[1][0] = 1.0; ra[1][1] = 0.0; }
            for (int q = 0; q < 2; ++q) {
                if (ra[q][0] > ra[q][1]) continue;
                for (uint32_t t = az_lower(az, m, ra[q][0]); t < m && az[t].phi <= ra[q][1]; ++t)
                    cand[nc++] = az[t].h;
            }
            qsort(cand, nc, sizeof(uint32_t), u32_cmp);
            for (uint32_t t = 0; t < nc; ++t) {
                const uint32_t o = cand[t];
                if (t && o == cand[t - 1]) continue;          /* (overlapping ranges) */
                if (orc_doublet_pass(x[i], y[i], x[o], y[o], P->cos_phi_window))
                    if (push(ci, i) || push(co, o)) goto out;
            }
        }
    }
    rc = 0;
out:
    free(az);
    free(cand);
    return rc;
}

/* Returns NULL on allocation failure or invalid input.  stage: 1 = stop after doublets,
 * 2 = after edges, 3 = after ntuplets, 4 = with fits.  windowed: doublets by the windowed search
 * (same cells, same order) instead of all pairs. */
orc_result *orc_reconstruct_w(uint32_t n, const float *xf, const float *yf, const float *zf,
                              const uint16_t *layer, const orc_params *P, int stage,
                              int windowed);

orc_result *orc_reconstruct(uint32_t n, const float *xf, const float *yf, const float *zf,
                            const uint16_t *layer, const orc_params *P, int stage)
{
    return orc_reconstruct_w(n, xf, yf, zf, layer, P, stage, 0);
}

orc_result *orc_reconstruct_w(uint32_t n, const float *xf, const float *yf, const float *zf,
                              const uint16_t *layer, const orc_params *P, int stage,
                              int windowed)
{
    orc_result *R = (orc_result *)calloc(1, sizeof(orc_result));
    double *x = NULL, *y = NULL, *z = NULL, *r = NULL;
    uint32_t *first = NULL, *cnt = NULL, *order = NULL, *nfirst = NULL;
    u32vec ci = {0}, co = {0}, ea = {0}, eb = {0};
    if (!R) return NULL;
    R->n_hits = n;
    if (P->max_hits > ORC_MAXH || P->min_hits < 2 || P->n_layers > ORC_MAX_LAYERS ||
        P->n_pairs > ORC_MAX_PAIRS)
        goto fail;
    for (uint32_t h = 0; h < n; ++h)
        if (layer[h] >= P->n_layers) goto fail;
    x = (double *)malloc((n + 1) * sizeof(double));
    y = (double *)malloc((n + 1) * sizeof(double));
    z = (double *)malloc((n + 1) * sizeof(double));
    r = (double *)malloc((n + 1) * sizeof(double));
    if (!x || !y || !z || !r) goto fail;
    for (uint32_t h = 0; h < n; ++h) {
        x[h] = (double)xf[h]; y[h] = (double)yf[h]; z[h] = (double)zf[h];
        r[h] = orc_radius(x[h], y[h]);
    }

    /* doublets: all pairs of every allowed layer pair (or the windowed search) */
    if (windowed) {
        if (doublets_windowed(n, x, y, layer, P, &ci, &co)) goto fail;
    } else for (uint32_t p = 0; p < P->n_pairs; ++p) {
        uint32_t Li = P->pair_inner[p], Lo = P->pair_outer[p];
        for (uint32_t i = 0; i < n; ++i) {
            if (layer[i] != Li) continue;
            for (uint32_t o = 0; o < n; ++o) {
                if (layer[o] != Lo) continue;
                if (orc_doublet_pass(x[i], y[i], x[o], y[o], P->cos_phi_window)) {
                    if (push(&ci, i) || push(&co, o)) goto fail;
                }
            }
        }
    }
    R->n_cells = (uint32_t)ci.n;
    R->cell_in = ci.a; R->cell_out = co.a;
    ci.a = co.a = NULL;
    if (stage <= 1) goto done;

    /* index of cells by inner hit (counting sort, cell order kept inside each hit) */
    first = (uint32_t *)calloc(n + 1, sizeof(uint32_t));
    cnt = (uint32_t *)calloc(n + 1, sizeof(uint32_t));
    order = (uint32_t *)malloc((R->n_cells + 1) * sizeof(uint32_t));
    if (!first || !cnt || !order) goto fail;
    for (uint32_t c = 0; c < R->n_cells; ++c) cnt[R->cell_in[c]]++;
    for (uint32_t h = 0; h < n; ++h) first[h + 1] = first[h] + cnt[h];
    memset(cnt, 0, (n + 1) * sizeof(uint32_t));
    for (uint32_t c = 0; c < R->n_cells; ++c) {
        uint32_t h = R->cell_in[c];
        order[first[h] + cnt[h]++] = c;
    }

    /* CA edges: A = (i, j), B = (j, k) */
    for (uint32_t A = 0; A < R->n_cells; ++A) {
        uint32_t i = R->cell_in[A], j = R->cell_out[A];
        for (uint32_t t = first[j]; t < first[j + 1]; ++t) {
            uint32_t B = order[t];
            uint32_t k = R->cell_out[B];
            if (!orc_theta_pass(r[i], z[i], r[j], z[j], r[k], z[k], P->theta_cut)) continue;
            if (!orc_dca_pass(x[i], y[i], x[j], y[j], x[k], y[k], P->dca_cut)) continue;
            if (push(&ea, A) || push(&eb, B)) goto fail;
        }
    }
    R->n_edges = (uint32_t)ea.n;
    R->edge_a = ea.a; R->edge_b = eb.a;
    ea.a = eb.a = NULL;
    if (stage <= 2) goto done;

    /* out-edges per cell, in edge order */
    nfirst = (uint32_t *)calloc(R->n_cells + 2, sizeof(uint32_t));
    uint32_t *nbr = (uint32_t *)malloc((R->n_edges + 1) * sizeof(uint32_t));
    uint32_t *ncnt = (uint32_t *)calloc(R->n_cells + 1, sizeof(uint32_t));
    if (!nfirst || !nbr || !ncnt) { free(nbr); free(ncnt); goto fail; }
    for (uint32_t e = 0; e < R->n_edges; ++e) ncnt[R->edge_a[e]]++;
    for (uint32_t c = 0; c < R->n_cells; ++c) nfirst[c + 1] = nfirst[c] + ncnt[c];
    memset(ncnt, 0, (R->n_cells + 1) * sizeof(uint32_t));
    for (uint32_t e = 0; e < R->n_edges; ++e) {
        uint32_t a = R->edge_a[e];
        nbr[nfirst[a] + ncnt[a]++] = R->edge_b[e];
    }
    free(ncnt);

    /* ntuplets: walk from every root cell */
    dfs_ctx d;
    memset(&d, 0, sizeof(d));
    d.P = P; d.cell_in = R->cell_in; d.cell_out = R->cell_out;
    d.nbr_first = nfirst; d.nbr = nbr; d.layer = layer;
    for (uint32_t c = 0; c < R->n_cells; ++c) {
        uint32_t path[ORC_MAXH];
        if (!((P->root_mask >> layer[R->cell_in[c]]) & 1u)) continue;
        path[0] = c;
        walk(&d, path, 1);
    }
    free(nbr);
    if (d.fail) { free(d.tup.a); free(d.tup_n.a); goto fail; }

    uint32_t ne = (uint32_t)d.tup_n.n;
    uint8_t *keep = (uint8_t *)malloc(ne + 1);
    if (!keep) { free(d.tup.a); free(d.tup_n.a); goto fail; }
    memset(keep, 1, ne + 1);
    if (P->drop_suffixes && ne > 0) {
        /* remove every emitted path that is a strict suffix of another emitted path */
        uint32_t *idx = (uint32_t *)malloc(ne * sizeof(uint32_t));
        if (!idx) { free(keep); free(d.tup.a); free(d.tup_n.a); goto fail; }
        for (uint32_t t = 0; t < ne; ++t) idx[t] = t;
        g_rows = d.tup.a;
        qsort(idx, ne, sizeof(uint32_t), idx_cmp);
        for (uint32_t t = 0; t < ne; ++t) {
            const uint32_t *Q = d.tup.a + (size_t)t * ORC_MAXH;
            uint32_t nq = d.tup_n.a[t];
            for (uint32_t k = 1; k + 2 <= nq; ++k) {
                uint32_t suf[ORC_MAXH];
                for (int i = 0; i < ORC_MAXH; ++i) suf[i] = 0xFFFFFFFFu;
                for (uint32_t i = k; i < nq; ++i) suf[i - k] = Q[i];
                /* binary search among the sorted rows */
                uint32_t lo = 0, hi = ne;
                while (lo < hi) {
                    uint32_t mid = (lo + hi) / 2;
                    int cmp = row_cmp(d.tup.a + (size_t)idx[mid] * ORC_MAXH, suf);
                    if (cmp < 0) lo = mid + 1; else hi = mid;
                }
                while (lo < ne && row_cmp(d.tup.a + (size_t)idx[lo] * ORC_MAXH, suf) == 0) {
                    keep[idx[lo]] = 0;
                    ++lo;
                }
            }
        }
        free(idx);
    }
    uint32_t nk = 0;
    for (uint32_t t = 0; t < ne; ++t) nk += keep[t];
    R->n_tuples = nk;
    R->tup_n = (uint8_t *)malloc(nk + 1);
    R->tup_hits = (uint32_t *)malloc(((size_t)nk + 1) * ORC_MAXH * sizeof(uint32_t));
    if (!R->tup_n || !R->tup_hits) { free(keep); free(d.tup.a); free(d.tup_n.a); goto fail; }
    for (uint32_t t = 0, o = 0; t < ne; ++t) {
        if (!keep[t]) continue;
        R->tup_n[o] = (uint8_t)d.tup_n.a[t];
        memcpy(R->tup_hits + (size_t)o * ORC_MAXH, d.tup.a + (size_t)t * ORC_MAXH,
               ORC_MAXH * sizeof(uint32_t));
        ++o;
    }
    free(keep); free(d.tup.a); free(d.tup_n.a);
    if (stage <= 3) goto done;

    /* fits */
    R->fit = (orc_track *)calloc(nk + 1, sizeof(orc_track));
    if (!R->fit) goto fail;
    for (uint32_t t = 0; t < nk; ++t) {
        double X[ORC_MAXH], Y[ORC_MAXH], Zz[ORC_MAXH];
        uint16_t L[ORC_MAXH];
        int nh = R->tup_n[t];
        for (int i = 0; i < nh; ++i) {
            uint32_t h = R->tup_hits[(size_t)t * ORC_MAXH + i];
            X[i] = x[h]; Y[i] = y[h]; Zz[i] = z[h]; L[i] = layer[h];
        }
        orc_fit_one(nh, X, Y, Zz, L, P, &R->fit[t]);
    }

done:
    free(x); free(y); free(z); free(r); free(first); free(cnt); free(order); free(nfirst);
    return R;
fail:
    free(x); free(y); free(z); free(r); free(first); free(cnt); free(order); free(nfirst);
    free(ci.a); free(co.a); free(ea.a); free(eb.a);
    orc_free(R);
    return NULL;
}
