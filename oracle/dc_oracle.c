/*
 * dc_oracle.c -- plain FP64 CPU oracle for the hybrid boundary-integral
 * diffusion-curve method (Bang, Serkh, Stein, Jacobson, TOG 42(6) 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path.  Everything is straightforward double-precision loops over
 * the definitions; OpenMP only splits independent target rows.
 *
 * What is computed (each function cites the passage it follows):
 *   - Gauss-Legendre rules by Newton on the Legendre recurrence (Sec. 3.3,
 *     Eq. 8-11: nodes and Legendre interpolation).
 *   - Cubic Bezier geometry and arc-length parametrisation by Newton on
 *     L(t) = T with L evaluated by Gauss-Legendre quadrature (App. B).
 *   - The hybrid discretisation: panels, Gauss-Legendre nodes placed in arc
 *     length, s equal-arc-length BEM segments per panel (Sec. 4.2, App. A/B),
 *     collocation points on the solve polyline (reading: App. C.1 treats a
 *     node lying on a segment as a singular integral for that segment).
 *   - Closed-form segment integrals of G and F (App. D, Eq. 50-53; the
 *     printed Eq. 50/51 are garbled, so the antiderivatives are written out
 *     from the integrands), scaled by arc length / chord length (App. A).
 *   - Dense hybrid operator rows A = Gbar * blockdiag(Pbar Pring^-1)
 *     (Eq. 19, Eq. 27) and the direct-sum layer potential at any points
 *     (Eq. 23 evaluated with the BEM-like sum of Eq. 17).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288
#define ORC_TWO_PI (2.0 * ORC_PI)

/* ------------------------------------------------------------------ misc */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ----------------------------------------------------- Legendre / Gauss */
/* Values P_0..P_{n-1} at x by the three-term recurrence. */
void orc_legendre_values(int n, double x, double *P)
{
    if (n <= 0) return;
    P[0] = 1.0;
    if (n == 1) return;
    P[1] = x;
    for (int k = 1; k + 1 < n; ++k)
        P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
}

/* P_n(z) and P_{n-1}(z) by the recurrence (n >= 1). */
static void legendre_pair(int n, double z, double *pn, double *pnm1)
{
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pnm1 = p0;
}

/* n-point Gauss-Legendre rule on [-1,1], nodes ascending.  Newton on P_n
 * from the start cos(pi (i + 3/4) / (n + 1/2)); P_n' from
 * P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1); w = 2 / ((1 - z^2) P_n'(z)^2). */
int orc_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return -1;
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), pn, pm, dp;
        for (int it = 0; it < 100; ++it) {
            legendre_pair(n, z, &pn, &pm);
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        legendre_pair(n, z, &pn, &pm);
        dp = n * (z * pn - pm) / (z * z - 1.0);
        x[n - 1 - i] = z;   /* the start values run from +1 down to -1 */
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* ------------------------------------------------------- Bezier (App. B) */
/* c = {x0,y0,x1,y1,x2,y2,x3,y3}; B(t) in Bernstein form. */
static void bez_point(const double *c, double t, double *px, double *py)
{
    double u = 1.0 - t;
    double b0 = u * u * u, b1 = 3.0 * t * u * u, b2 = 3.0 * t * t * u, b3 = t * t * t;
    *px = b0 * c[0] + b1 * c[2] + b2 * c[4] + b3 * c[6];
    *py = b0 * c[1] + b1 * c[3] + b2 * c[5] + b3 * c[7];
}

static double bez_speed(const double *c, double t)
{
    double u = 1.0 - t;
    double dx = 3.0 * (u * u * (c[2] - c[0]) + 2.0 * t * u * (c[4] - c[2]) + t * t * (c[6] - c[4]));
    double dy = 3.0 * (u * u * (c[3] - c[1]) + 2.0 * t * u * (c[5] - c[3]) + t * t * (c[7] - c[5]));
    return sqrt(dx * dx + dy * dy);
}

#define ORC_ALQ_N 20     /* points of the arc-length quadrature rule   */
#define ORC_ALQ_SUB 32   /* equal sub-intervals of [0, t]              */
static double g_alq_x[ORC_ALQ_N], g_alq_w[ORC_ALQ_N];
static int g_alq_ready = 0;

static void alq_init(void)
{
    if (!g_alq_ready) {
        orc_gauss_legendre(ORC_ALQ_N, g_alq_x, g_alq_w);
        g_alq_ready = 1;
    }
}

/* L(t) = int_0^t |B'(tau)| dtau by composite Gauss-Legendre (App. B). */
double orc_arclen(const double *c, double t)
{
    alq_init();
    double h = t / ORC_ALQ_SUB, acc = 0.0;
    for (int j = 0; j < ORC_ALQ_SUB; ++j) {
        double a = j * h, mid = a + 0.5 * h, part = 0.0;
        for (int i = 0; i < ORC_ALQ_N; ++i)
            part += g_alq_w[i] * bez_speed(c, mid + 0.5 * h * g_alq_x[i]);
        acc += 0.5 * h * part;
    }
    return acc;
}

/* Parameter t with L(t) = T: Newton's update t <- t - (L(t) - T) / L'(t),
 * L'(t) = |B'(t)| (App. B), kept inside a bisection bracket. */
double orc_t_of_s(const double *c, double T, double Ltot)
{
    if (T <= 0.0) return 0.0;
    if (T >= Ltot) return 1.0;
    double lo = 0.0, hi = 1.0, t = T / Ltot;
    for (int it = 0; it < 200; ++it) {
        double f = orc_arclen(c, t) - T;
        if (fabs(f) <= 1e-15 * Ltot) break;
        if (f > 0) hi = t; else lo = t;
        double tn = t - f / bez_speed(c, t);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        if (fabs(tn - t) < 1e-17) { t = tn; break; }
        t = tn;
    }
    return t;
}

/* ------------------------------------------------------- discretisation */
/*
 * Discretise a drawing (Sec. 4.2 with App. A/B):
 *   panel j of curve i covers arc lengths [f_j L_i, f_{j+1} L_i]; g nodes at
 *   arc length s = a + (b - a)(x_m + 1)/2 (x_m Gauss-Legendre on [-1,1]);
 *   nseg segments per panel with vertices at equal arc length.
 * Outputs (caller-allocated, P = total panels, N = P g, S = P nseg):
 *   node_xy[N][2]   collocation point on the solve polyline
 *   node_t[N]       Bezier parameter of the node (for the boundary colours)
 *   node_seg[N]     global index of the segment holding the node
 *   node_seg2[N]    second segment when the node sits on a vertex, else -1
 *   node_curve[N]
 *   seg_xy[S][4]    x1,y1,x2,y2
 *   seg_w[S]        arc length / chord length of the segment (App. A)
 *   curve_len[n]
 * Returns 0 on success.
 */
int orc_discretise(int n_curves, const double *ctrl, const int *panel_ptr,
                   const double *panel_start, int g, int nseg,
                   double *node_xy, double *node_t, int *node_seg,
                   int *node_seg2, int *node_curve, double *seg_xy,
                   double *seg_w, double *curve_len)
{
    double *gx = (double *)malloc(sizeof(double) * g);
    double *gw = (double *)malloc(sizeof(double) * g);
    if (!gx || !gw) { free(gx); free(gw); return -1; }
    orc_gauss_legendre(g, gx, gw);
    alq_init();   /* before the threads start */
    int err = 0;
#pragma omp parallel for schedule(dynamic)
    for (int ci = 0; ci < n_curves; ++ci) {
        const double *c = ctrl + 8 * ci;
        double L = orc_arclen(c, 1.0);
        curve_len[ci] = L;
        int p0 = panel_ptr[ci], p1 = panel_ptr[ci + 1];
        for (int pj = p0; pj < p1; ++pj) {
            double fa = panel_start[pj];
            double fb = (pj + 1 < p1) ? panel_start[pj + 1] : 1.0;
            double sa = fa * L, sb = fb * L, h = (sb - sa) / nseg;
            /* vertices */
            double *vx = (double *)malloc(sizeof(double) * (nseg + 1));
            double *vy = (double *)malloc(sizeof(double) * (nseg + 1));
            for (int k = 0; k <= nseg; ++k) {
                double s = (k == nseg) ? sb : sa + k * h;
                double t = (k == nseg && fb == 1.0) ? 1.0 : orc_t_of_s(c, s, L);
                if (k == 0 && fa == 0.0) t = 0.0;
                bez_point(c, t, &vx[k], &vy[k]);
            }
            for (int k = 0; k < nseg; ++k) {
                int sidx = pj * nseg + k;
                double *q = seg_xy + 4 * (size_t)sidx;
                q[0] = vx[k]; q[1] = vy[k]; q[2] = vx[k + 1]; q[3] = vy[k + 1];
                double chord = hypot(vx[k + 1] - vx[k], vy[k + 1] - vy[k]);
                seg_w[sidx] = h / chord;
            }
            /* nodes */
            for (int m = 0; m < g; ++m) {
                int nidx = pj * g + m;
                double u = 0.5 * (gx[m] + 1.0) * nseg;   /* position in segment units */
                int k = (int)floor(u);
                if (k >= nseg) k = nseg - 1;
                double tau = u - k;
                int alt = -1;
                if (tau < 1e-12 && k > 0) alt = pj * nseg + k - 1;
                if (tau > 1.0 - 1e-12 && k + 1 < nseg) alt = pj * nseg + k + 1;
                node_xy[2 * nidx] = vx[k] + tau * (vx[k + 1] - vx[k]);
                node_xy[2 * nidx + 1] = vy[k] + tau * (vy[k + 1] - vy[k]);
                node_seg[nidx] = pj * nseg + k;
                node_seg2[nidx] = alt;
                node_curve[nidx] = ci;
                double s_node = sa + 0.5 * (gx[m] + 1.0) * (sb - sa);
                node_t[nidx] = orc_t_of_s(c, s_node, L);
            }
            free(vx);
            free(vy);
        }
    }
    free(gx);
    free(gw);
    return err;
}

/* -------------------------------------------- closed-form segment rules */
/*
 * Integrals over the straight chord p1 -> p2 of
 *   G(p,q) = -log|p - q| / (2 pi)                         (Eq. 3)
 *   F(p,q) = -(p - q).n(p) / (2 pi |p - q|^2)             (Eq. 4)
 * with n the right-hand unit normal (t_y, -t_x) of the chord direction t.
 * In the chord frame, s runs along t from s1 to s2 (endpoint coordinates
 * relative to the foot of q) and h = (p1 - q).n is the constant offset:
 *   int log|p-q| dS = [ s log sqrt(s^2+h^2) - s + h atan(s/h) ]_{s1}^{s2}
 *   int (q-p).n/|q-p|^2 dS = -h int ds/(s^2+h^2) = -[ atan(s/h) ]_{s1}^{s2}
 * (App. D; the printed Eq. 50/51 are garbled and are not used).  When q lies
 * on the chord the singular forms of Eq. 52 and Eq. 53 apply:
 *   int G dS = (c - e1 log e1 - e2 log e2) / (2 pi),   int F dS = 0.
 */
static double xlogr(double s, double r)
{
    return (r > 0.0) ? s * log(r) : 0.0;
}

void orc_segment_GF(double x1, double y1, double x2, double y2, double qx,
                    double qy, int singular, double *G, double *F)
{
    double dx = x2 - x1, dy = y2 - y1;
    double c = sqrt(dx * dx + dy * dy);
    if (singular) {
        double e1 = hypot(qx - x1, qy - y1), e2 = hypot(qx - x2, qy - y2);
        *G = (c - xlogr(e1, e1) - xlogr(e2, e2)) / ORC_TWO_PI;
        *F = 0.0;
        return;
    }
    double tx = dx / c, ty = dy / c;
    double ax = x1 - qx, ay = y1 - qy, bx = x2 - qx, by = y2 - qy;
    double s1 = ax * tx + ay * ty, s2 = bx * tx + by * ty;
    double h = ax * ty - ay * tx;
    double r1 = sqrt(ax * ax + ay * ay), r2 = sqrt(bx * bx + by * by);
    double dang = (h != 0.0) ? atan(s2 / h) - atan(s1 / h) : 0.0;
    double ilog = xlogr(s2, r2) - xlogr(s1, r1) - (s2 - s1) + h * dang;
    *G = -ilog / ORC_TWO_PI;
    *F = -dang / ORC_TWO_PI;
}

/* ------------------------------------------------- dense hybrid rows */
/*
 * Rows of the hybrid operators for n_t targets (Eq. 19 and its F analogue):
 *   AG[i][j g + m] = sum_k w_k int_{S_jk} G(p, q_i) dS * Lambda[k][m]
 * where k runs over the nseg segments of panel j and Lambda = Pbar Pring^-1
 * (nseg x g, identical for every panel because segments are equal in arc
 * length).  tgt_seg / tgt_seg2 mark the singular segment(s) of each target
 * (-1 for none).  AG and AF are n_t x (P g), row-major.
 */
void orc_hybrid_rows(int n_t, const double *tgt_xy, const int *tgt_seg,
                     const int *tgt_seg2, int n_panels, int nseg, int g,
                     const double *seg_xy, const double *seg_w,
                     const double *Lambda, double *AG, double *AF)
{
    int ncol = n_panels * g;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < n_t; ++i) {
        double qx = tgt_xy[2 * i], qy = tgt_xy[2 * i + 1];
        double *rg = AG + (size_t)i * ncol, *rf = AF + (size_t)i * ncol;
        memset(rg, 0, sizeof(double) * ncol);
        memset(rf, 0, sizeof(double) * ncol);
        for (int pj = 0; pj < n_panels; ++pj) {
            for (int k = 0; k < nseg; ++k) {
                int sidx = pj * nseg + k;
                const double *q = seg_xy + 4 * (size_t)sidx;
                int sing = (sidx == tgt_seg[i]) || (sidx == tgt_seg2[i]);
                double G, F;
                orc_segment_GF(q[0], q[1], q[2], q[3], qx, qy, sing, &G, &F);
                G *= seg_w[sidx];
                F *= seg_w[sidx];
                const double *lam = Lambda + (size_t)k * g;
                for (int m = 0; m < g; ++m) {
                    rg[pj * g + m] += G * lam[m];
                    rf[pj * g + m] += F * lam[m];
                }
            }
        }
    }
}

/*
 * Direct-sum layer potential (Eq. 23 with the BEM-like sum over segments):
 *   u_c(x) = sum_k w_k [ sigma_bar[k][c] int G + mu_bar[k][c] int F ],
 * c = 0..2.  tgt_seg / tgt_seg2 may be NULL (no singular segments).
 */
void orc_layer_potential(int n_t, const double *tgt_xy, const int *tgt_seg,
                         const int *tgt_seg2, int n_seg, const double *seg_xy,
                         const double *seg_w, const double *sigma_bar,
                         const double *mu_bar, double *u)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n_t; ++i) {
        double qx = tgt_xy[2 * i], qy = tgt_xy[2 * i + 1];
        double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
        int s1 = tgt_seg ? tgt_seg[i] : -1, s2 = tgt_seg2 ? tgt_seg2[i] : -1;
        for (int k = 0; k < n_seg; ++k) {
            const double *q = seg_xy + 4 * (size_t)k;
            double G, F;
            orc_segment_GF(q[0], q[1], q[2], q[3], qx, qy, k == s1 || k == s2, &G, &F);
            G *= seg_w[k];
            F *= seg_w[k];
            acc0 += G * sigma_bar[3 * k + 0] + F * mu_bar[3 * k + 0];
            acc1 += G * sigma_bar[3 * k + 1] + F * mu_bar[3 * k + 1];
            acc2 += G * sigma_bar[3 * k + 2] + F * mu_bar[3 * k + 2];
        }
        u[3 * i + 0] = acc0;
        u[3 * i + 1] = acc1;
        u[3 * i + 2] = acc2;
    }
}
