// Adaptive subdivision and local re-solve (Sec. 6.1 and 6.3, Alg. 5-7):
// the device kernels.  The host logic (split decisions, the rebuilt
// discretisation, the labels and the masked GMRES) is in dc_api.cpp.
//
//  * legendre_top_kernel: per panel, the highest-order Legendre coefficient
//    of the density, c_{g-1} = sum_m q_m sigma_m with q the last row of the
//    inverse of the Legendre Vandermonde matrix at the Gauss-Legendre nodes
//    (Alg. 5's test), as the maximum of |c_{g-1}| over the colour channels.
//  * split_interp_kernel: the warm start of Sec. 6.1 -- each panel of the
//    refined discretisation takes E_t sigma_old(panel) with E_0 = I (panel
//    kept), E_1 / E_2 the old panel's Legendre expansion evaluated at the
//    nodes of its left / right half.
//  * unit_density_kernel: rho = 1 on the nodes of up to three panels, one
//    per colour channel (Eq. 40's FMM of a unit density, three panels per
//    operator application), 0 elsewhere.
//  * panel_range_kernel: max - min of a potential over each panel's nodes
//    per channel (the two sides of Eq. 41).
//  * node_mask_kernel: zeroes node values outside a per-panel mask (the
//    restriction to the re-solving panels of the local system).
//  * blend_kernel: node values taken from one vector or another by a
//    per-panel mask, each scaled (the Dirichlet / Neumann parts of the mixed
//    problem of Sec. 4.3 and its block-diagonal preconditioner).
#include <cuda_runtime.h>

#include <vector>

#include "dc_internal.h"

namespace dc {
namespace {

constexpr int kThreads = 256;

__global__ void legendre_top_kernel(const double *__restrict__ sigma, int n_panels, int g,
                                    const double *__restrict__ q, double *__restrict__ top) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_panels) return;
    double m = 0.0;
    for (int c = 0; c < 3; ++c) {
        double a = 0.0;
        for (int k = 0; k < g; ++k) a += q[k] * sigma[3 * ((size_t)p * g + k) + c];
        m = fmax(m, fabs(a));
    }
    top[p] = m;
}

__global__ void split_interp_kernel(const double *__restrict__ sig_old, const int2 *__restrict__ pmap,
                                    const double *__restrict__ E, int g, int n_new, double *__restrict__ sig_new) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;   // (new node, channel)
    if (t >= 3 * n_new * g) return;
    const int c = t % 3, node = t / 3, p = node / g, n = node - p * g;
    const int2 pm = pmap[p];
    const double *e = E + ((size_t)pm.y * g + n) * g;
    const double *s = sig_old + 3 * (size_t)pm.x * g + c;
    double a = 0.0;
    for (int m = 0; m < g; ++m) a += e[m] * s[3 * m];
    sig_new[t] = a;
}

__global__ void unit_density_kernel(double *__restrict__ x, int N, int g, int p0, int p1, int p2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * N) return;
    const int c = t % 3, p = (t / 3) / g;
    const int want = c == 0 ? p0 : (c == 1 ? p1 : p2);
    x[t] = (p == want) ? 1.0 : 0.0;
}

__global__ void panel_range_kernel(const double *__restrict__ v, int n_panels, int g, double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;   // (panel, channel)
    if (t >= 3 * n_panels) return;
    const int c = t % 3, p = t / 3;
    const double *a = v + 3 * (size_t)p * g + c;
    double lo = a[0], hi = a[0];
    for (int m = 1; m < g; ++m) {
        lo = fmin(lo, a[3 * m]);
        hi = fmax(hi, a[3 * m]);
    }
    out[t] = hi - lo;
}

// out = max |a - b| over n values (a FP32, b FP64), as the bits of a
// non-negative float (their integer order is the float order)
__global__ void max_diff_kernel(const float *__restrict__ a, const double *__restrict__ b, long long n,
                                unsigned *__restrict__ out) {
    float m = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, (float)fabs((double)a[i] - b[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// out = pmask[panel] ? beta b : alpha a at every node and channel
__global__ void blend_kernel(double *__restrict__ out, const double *__restrict__ a, double alpha,
                             const double *__restrict__ b, double beta, const unsigned char *__restrict__ pmask,
                             int N, int g) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * N) return;
    out[t] = pmask[(t / 3) / g] ? beta * b[t] : alpha * a[t];
}

__global__ void node_mask_kernel(double *__restrict__ v, const unsigned char *__restrict__ pmask, int N, int g) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * N) return;
    if (!pmask[(t / 3) / g]) v[t] = 0.0;
}

inline int blocks(long long n) { return int((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_legendre_top(const double *sigma, int n_panels, int g, const double *q, double *top,
                                cudaStream_t st) {
    if (n_panels <= 0) return cudaSuccess;
    legendre_top_kernel<<<blocks(n_panels), kThreads, 0, st>>>(sigma, n_panels, g, q, top);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_split_interp(const double *sig_old, const int2 *pmap, const double *E, int g, int n_new,
                                double *sig_new, cudaStream_t st) {
    if (n_new <= 0) return cudaSuccess;
    split_interp_kernel<<<blocks(3LL * n_new * g), kThreads, 0, st>>>(sig_old, pmap, E, g, n_new, sig_new);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_unit_density(double *x, int N, int g, const int panels[3], cudaStream_t st) {
    unit_density_kernel<<<blocks(3LL * N), kThreads, 0, st>>>(x, N, g, panels[0], panels[1], panels[2]);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_panel_range(const double *v, int n_panels, int g, double *out, cudaStream_t st) {
    panel_range_kernel<<<blocks(3LL * n_panels), kThreads, 0, st>>>(v, n_panels, g, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_max_diff(const float *a, const double *b, long long n, unsigned *out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    max_diff_kernel<<<4 * 152, kThreads, 0, st>>>(a, b, n, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_blend(double *out, const double *a, double alpha, const double *b, double beta,
                         const unsigned char *pmask, int N, int g, cudaStream_t st) {
    blend_kernel<<<blocks(3LL * N), kThreads, 0, st>>>(out, a, alpha, b, beta, pmask, N, g);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_node_mask(double *v, const unsigned char *pmask, int N, int g, cudaStream_t st) {
    node_mask_kernel<<<blocks(3LL * N), kThreads, 0, st>>>(v, pmask, N, g);
    note_launch();
    return cudaGetLastError();
}

}  // namespace dc

namespace dc {
namespace {

// P_0..P_{n-1} at x by the three-term recurrence (k + 1) P_{k+1} =
// (2k + 1) x P_k - k P_{k-1}.
void legendre_row(int n, double x, double *P) {
    if (n <= 0) return;
    P[0] = 1.0;
    if (n > 1) P[1] = x;
    for (int k = 1; k + 1 < n; ++k) P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
}

// T[k][m] = (2k + 1)/2 w_m P_k(x_m): the discrete Legendre transform at the
// g Gauss-Legendre nodes, c_k = sum_m T[k][m] sigma_m, exact for densities
// that are polynomials of degree < g (the quadrature integrates P_j P_k
// exactly for j + k <= 2g - 1), so T inverts the Vandermonde matrix.
std::vector<double> legendre_transform(int g) {
    std::vector<double> x(g), w(g), P(g), T((size_t)g * g);
    gauss_legendre_rule(g, x.data(), w.data());
    for (int m = 0; m < g; ++m) {
        legendre_row(g, x[m], P.data());
        for (int k = 0; k < g; ++k) T[(size_t)k * g + m] = 0.5 * (2.0 * k + 1.0) * w[m] * P[k];
    }
    return T;
}

}  // namespace

void legendre_top_row(int g, double *q) {
    const std::vector<double> T = legendre_transform(g);
    for (int m = 0; m < g; ++m) q[m] = T[(size_t)(g - 1) * g + m];
}

void split_matrices(int g, double *E) {
    const std::vector<double> T = legendre_transform(g);
    std::vector<double> x(g), w(g), P(g);
    gauss_legendre_rule(g, x.data(), w.data());
    for (int t = 0; t < 3; ++t)
        for (int n = 0; n < g; ++n) {
            double *e = E + ((size_t)t * g + n) * g;
            if (t == 0) {
                for (int m = 0; m < g; ++m) e[m] = (m == n) ? 1.0 : 0.0;
                continue;
            }
            // node n of the left (t = 1) or right (t = 2) half, in the old
            // panel's coordinate on [-1, 1] (arc length is linear in both)
            const double xo = t == 1 ? 0.5 * (x[n] - 1.0) : 0.5 * (x[n] + 1.0);
            legendre_row(g, xo, P.data());
            for (int m = 0; m < g; ++m) {
                double a = 0.0;
                for (int k = 0; k < g; ++k) a += P[k] * T[(size_t)k * g + m];
                e[m] = a;
            }
        }
}

}  // namespace dc
