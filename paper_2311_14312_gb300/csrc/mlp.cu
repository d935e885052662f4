// Learned warm start for GMRES: a small MLP (n_in -> H -> H -> H -> n_out,
// GELU) that predicts a panel's scaled density (sigma * panel length at its
// g nodes, one colour channel) from local features.  Not part of the paper,
// whose warm start re-interpolates an old solution (Sec. 6.1); here the
// network is trained on densities the solver itself produced.
//
// Parameters are FP32 masters packed layer by layer (W_l [out][in], then
// b_l [out]); the forward and backward passes read BF16-rounded weights and
// accumulate in FP32.  All products go through one tcgen05 GEMM (mlp_tc.cuh:
// TF32 terms, BF16 weights exact, FP32 operands split in two) with an
// optional bias + GELU epilogue; reductions over the batch run inside the
// GEMM in a fixed order (deterministic).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "dc_internal.h"
#include "mlp_tc.cuh"

namespace dc {
namespace mlp {

constexpr int kLayers = 4;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    // d/dx [x Phi(x)] = Phi(x) + x phi(x)
    const float phi = 0.39894228040143268f * __expf(-0.5f * x * x);
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * phi;
}

__global__ void to_bf16_kernel(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16(a[i]);
}

// dY = 2 (Y - T) / (batch n_out); loss partials per block (fixed order)
__global__ void mse_kernel(const float *__restrict__ Y, const float *__restrict__ T, float *__restrict__ dY,
                           size_t n, float scale, float *__restrict__ partial) {
    __shared__ float red[256];
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f;
    if (i < n) {
        d = Y[i] - T[i];
        dY[i] = 2.f * d * scale;
    }
    red[threadIdx.x] = d * d;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void sum_kernel(const float *__restrict__ partial, int n, float scale, float *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += partial[i];
        *out = (float)(s * scale);
    }
}

// dZ = dY * gelu'(Zpre)
__global__ void gelu_back_kernel(const float *__restrict__ dY, const float *__restrict__ Z,
                                 float *__restrict__ dZ, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dZ[i] = dY[i] * gelu_grad(Z[i]);
}

// db[j] = sum_m dZ[m][j], fixed order over m
__global__ void colsum_kernel(const float *__restrict__ dZ, int M, int N, float *__restrict__ db) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += dZ[(size_t)m * N + j];
    db[j] = s;
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, size_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

struct Dims {
    int d[kLayers + 1];
    size_t woff[kLayers], boff[kLayers], total;
};

Dims dims(int n_in, int hidden, int n_out) {
    Dims D;
    D.d[0] = n_in;
    D.d[1] = D.d[2] = D.d[3] = hidden;
    D.d[4] = n_out;
    size_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        D.woff[l] = o;
        o += (size_t)D.d[l + 1] * D.d[l];
        D.boff[l] = o;
        o += D.d[l + 1];
    }
    D.total = o;
    return D;
}

// Workspace floats: BF16 weight copy (as floats/2, rounded up), per layer
// pre-activation and activation [batch][out], two gradient buffers, loss
// partials.
size_t workspace_floats(const Dims &D, int batch) {
    size_t w = (D.total + 1) / 2 + 8;
    for (int l = 0; l < kLayers; ++l) w += 2 * (size_t)batch * D.d[l + 1];
    size_t widest = 0;
    for (int l = 0; l <= kLayers; ++l) widest = widest > (size_t)D.d[l] ? widest : (size_t)D.d[l];
    w += 2 * (size_t)batch * widest;
    w += ((size_t)batch * D.d[kLayers] + 255) / 256 + 8;
    w += 8;   // the GEMMs' wait-limit flag
    return w;
}

// C[M][N] = op(A) op(B) (+ bias[N]) (GELU if act), FP32 accumulate.
//   opA = A [M][K] (lda) or, with ta, A^T of A [K][M]
//   opB = B^T of B [N][K] (ldb) or, with tb, B [K][N]
// B may be BF16 (weights) or FP32 (activations).
void gemm(cudaStream_t st, int M, int N, int K, const float *A, int lda, int ta, const void *B, int ldb,
          int tb, bool b_bf16, float *C, int ldc, const float *bias, int act, float *Zpre, int *err) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gemm_tc_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGtSmem);
        cudaFuncSetAttribute(gemm_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGtSmem);
        attr = true;
    }
    dim3 grid((M + kGtM - 1) / kGtM, (N + kGtN - 1) / kGtN);
    if (b_bf16)
        gemm_tc_kernel<__nv_bfloat16><<<grid, 128, kGtSmem, st>>>(M, N, K, A, lda, ta,
                                                                 static_cast<const __nv_bfloat16 *>(B), ldb, tb,
                                                                 C, ldc, bias, act, Zpre, err);
    else
        gemm_tc_kernel<float><<<grid, 128, kGtSmem, st>>>(M, N, K, A, lda, ta, static_cast<const float *>(B), ldb,
                                                         tb, C, ldc, bias, act, Zpre, err);
    note_launch();
}

}  // namespace mlp
}  // namespace dc

using namespace dc::mlp;

namespace {
struct Layout {
    __nv_bfloat16 *wbf;
    float *Z[kLayers], *Y[kLayers], *g0, *g1, *partial;
    int *err;   // set when a GEMM's wait on its MMAs ran out
};
Layout carve(const Dims &D, int batch, float *work) {
    Layout L;
    L.wbf = reinterpret_cast<__nv_bfloat16 *>(work);
    float *p = work + (D.total + 1) / 2 + 8;
    for (int l = 0; l < kLayers; ++l) {
        L.Z[l] = p;
        p += (size_t)batch * D.d[l + 1];
        L.Y[l] = p;
        p += (size_t)batch * D.d[l + 1];
    }
    size_t widest = 0;
    for (int l = 0; l <= kLayers; ++l) widest = widest > (size_t)D.d[l] ? widest : (size_t)D.d[l];
    L.g0 = p;
    p += (size_t)batch * widest;
    L.g1 = p;
    p += (size_t)batch * widest;
    L.partial = p;
    p += ((size_t)batch * D.d[kLayers] + 255) / 256 + 8;
    L.err = reinterpret_cast<int *>(p);
    return L;
}

// DC_ERR_TIMEOUT when a GEMM's wait on its MMAs ran out (the stream drained)
dc_status check_waits(const Layout &L, cudaStream_t st) {
    int flag = 0;
    if (cudaMemcpyAsync(&flag, L.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return DC_ERR_CUDA;
    return flag ? DC_ERR_TIMEOUT : DC_OK;
}

// forward; the output of the last layer is L.Y[3] (linear)
void forward(const Dims &D, const float *params, int batch, const float *x, const Layout &L,
             cudaStream_t st) {
    size_t n = D.total;
    cudaMemsetAsync(L.err, 0, sizeof(int), st);
    to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(params, L.wbf, n);
    dc::note_launch();
    const float *in = x;
    for (int l = 0; l < kLayers; ++l) {
        const int out = D.d[l + 1], inn = D.d[l];
        gemm(st, batch, out, inn, in, inn, 0, L.wbf + D.woff[l], inn, 0, true, L.Y[l], out,
             params + D.boff[l], l + 1 < kLayers ? 1 : 0, L.Z[l], L.err);
        in = L.Y[l];
    }
}
}  // namespace

extern "C" {

size_t dc_aux_mlp_param_count(int n_in, int hidden, int n_out) { return dims(n_in, hidden, n_out).total; }

size_t dc_aux_mlp_workspace_floats(int n_in, int hidden, int n_out, int batch) {
    return workspace_floats(dims(n_in, hidden, n_out), batch);
}

dc_status dc_aux_mlp_forward(int n_in, int hidden, int n_out, const float *params, int batch,
                             const float *x, float *y, float *work, void *stream) {
    if (n_in < 1 || hidden < 1 || n_out < 1 || batch < 0 || !params || (batch > 0 && (!x || !y || !work)))
        return DC_ERR_ARG;
    if (batch == 0) return DC_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Dims D = dims(n_in, hidden, n_out);
    Layout L = carve(D, batch, work);
    forward(D, params, batch, x, L, st);
    cudaError_t e = cudaMemcpyAsync(y, L.Y[kLayers - 1], sizeof(float) * (size_t)batch * n_out,
                                    cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return DC_ERR_CUDA;
    return check_waits(L, st);
}

dc_status dc_aux_mlp_loss_grad(int n_in, int hidden, int n_out, const float *params, int batch,
                               const float *x, const float *target, float *grad, float *loss,
                               float *work, void *stream) {
    if (n_in < 1 || hidden < 1 || n_out < 1 || batch < 1 || !params || !x || !target || !grad ||
        !loss || !work)
        return DC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Dims D = dims(n_in, hidden, n_out);
    Layout L = carve(D, batch, work);
    forward(D, params, batch, x, L, st);
    // loss = mean over batch and outputs of (y - t)^2
    size_t ny = (size_t)batch * n_out;
    int nb = (int)((ny + 255) / 256);
    float scale = 1.f / (float)ny;
    mse_kernel<<<nb, 256, 0, st>>>(L.Y[kLayers - 1], target, L.g0, ny, scale, L.partial);
    dc::note_launch();
    sum_kernel<<<1, 32, 0, st>>>(L.partial, nb, scale, loss);
    dc::note_launch();
    // backward: g0 holds dL/d(output of layer l) (pre-activation for the last)
    float *dcur = L.g0, *dnext = L.g1;
    for (int l = kLayers - 1; l >= 0; --l) {
        const int out = D.d[l + 1], inn = D.d[l];
        if (l + 1 < kLayers) {
            size_t n = (size_t)batch * out;
            gelu_back_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dcur, L.Z[l], dcur, n);
            dc::note_launch();
        }
        const float *xin = (l == 0) ? x : L.Y[l - 1];
        // dW [out][inn] = dZ^T [out][batch] x X [batch][inn]
        gemm(st, out, inn, batch, dcur, out, 1, xin, inn, 1, false, grad + D.woff[l], inn, nullptr, 0,
             nullptr, L.err);
        colsum_kernel<<<(out + 127) / 128, 128, 0, st>>>(dcur, batch, out, grad + D.boff[l]);
        dc::note_launch();
        if (l > 0) {
            // dX [batch][inn] = dZ [batch][out] x W [out][inn]
            gemm(st, batch, inn, out, dcur, out, 0, L.wbf + D.woff[l], inn, 1, true, dnext, inn, nullptr,
                 0, nullptr, L.err);
            float *t = dcur;
            dcur = dnext;
            dnext = t;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return DC_ERR_CUDA;
    return check_waits(L, st);
}

dc_status dc_aux_mlp_adam(size_t n, float *params, const float *grad, float *m, float *v, float lr,
                          float beta1, float beta2, float eps, int step, void *stream) {
    if (!params || !grad || !m || !v || step < 1) return DC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(params, grad, m, v, n, lr, beta1, beta2, eps,
                                                             c1, c2);
    dc::note_launch();
    return cudaGetLastError() == cudaSuccess ? DC_OK : DC_ERR_CUDA;
}

}  // extern "C"
