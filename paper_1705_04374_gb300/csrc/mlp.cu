// MLP surrogate for the OF-MLMC estimator's extra control variate.
//
// Network: d_in -> H (x n_hidden, exact-erf GELU) -> d_out, weights stored
// (fan_in x fan_out) row-major, one bias per output.  Inputs are standardised
// (x - mean) * inv_std inside the first GEMM's operand load; targets are
// standardised by the caller-supplied affine map, which forward undoes.
//
// Arithmetic: every GEMM rounds its operands to BF16 (round to nearest even)
// when it stages them in shared memory and accumulates in FP32 on the tensor
// cores (mma.sync m16n8k16 bf16 -> f32).  Master weights, activations,
// gradients and the Adam moments stay FP32.  Every reduction has a fixed
// order, so training is deterministic.
//
// Kernels: gemm_kernel (three operand layouts: X W, X^T dZ, dZ W^T, with
// bias / GELU epilogues), gelu_backward_kernel, column_sum_kernel (bias
// gradients), mse_kernel (loss and its gradient), adam_kernel, and the cloud
// feature builder (bubbles sorted by distance from the domain centre).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "ofmlmc.h"

using ofm::fail;

namespace {

constexpr int GBM = 64, GBN = 64, GBK = 32, GTHREADS = 128;
constexpr int SPAD = 8;  // bf16 padding per shared row (keeps rows 16-byte aligned, spreads banks)

__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, const unsigned* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2 };

// C[M x N] = op(A)[M x K] * op(B)[K x N] with BF16 operands, FP32 accumulation.
//   A(m, k) = TA ? A[k * lda + m] : A[m * lda + k]   (optionally (a - shift[f]) * scale[f],
//                                                      f = the feature index, k or m)
//   B(k, n) = TB ? B[n * ldb + k] : B[k * ldb + n]
// Epilogues: C = acc; C = acc + bias[n]; C = acc + bias[n] and H = gelu(C).
template <bool TA, bool TB>
__global__ void __launch_bounds__(GTHREADS) gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                        const float* __restrict__ B, int ldb, float* __restrict__ C,
                                                        int ldc, const float* __restrict__ bias, int epi,
                                                        float* __restrict__ H, const float* __restrict__ shift,
                                                        const float* __restrict__ scale) {
    __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + SPAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + SPAD];  // stored [n][k]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;

    for (int k0 = 0; k0 < K; k0 += GBK) {
        for (int idx = tid; idx < GBM * GBK; idx += GTHREADS) {
            int mm, kk;
            if (TA) {
                mm = idx % GBM;
                kk = idx / GBM;
            } else {
                kk = idx % GBK;
                mm = idx / GBK;
            }
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.0f;
            if (m < M && k < K) {
                v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
                if (shift) {
                    const int f = TA ? m : k;
                    v = (v - shift[f]) * scale[f];
                }
            }
            As[mm][kk] = __float2bfloat16_rn(v);
        }
        for (int idx = tid; idx < GBN * GBK; idx += GTHREADS) {
            int nn, kk;
            if (TB) {
                kk = idx % GBK;
                nn = idx / GBK;
            } else {
                nn = idx % GBN;
                kk = idx / GBN;
            }
            const int n = n0 + nn, k = k0 + kk;
            float v = 0.0f;
            if (n < N && k < K) v = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
            Bs[nn][kk] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GBK; ks += 16) {
            unsigned af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + g;
                af[i][0] = *reinterpret_cast<const unsigned*>(&As[r][ks + 2 * t]);
                af[i][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][ks + 2 * t]);
                af[i][2] = *reinterpret_cast<const unsigned*>(&As[r][ks + 2 * t + 8]);
                af[i][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][ks + 2 * t + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + g;
                bf[j][0] = *reinterpret_cast<const unsigned*>(&Bs[c][ks + 2 * t]);
                bf[j][1] = *reinterpret_cast<const unsigned*>(&Bs[c][ks + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm + i * 16 + g + (r >= 2 ? 8 : 0);
                const int n = n0 + wn + j * 8 + 2 * t + (r & 1);
                if (m < M && n < N) {
                    float v = acc[i][j][r];
                    if (epi != EPI_STORE) v += bias[n];
                    C[(size_t)m * ldc + n] = v;
                    if (epi == EPI_BIAS_GELU) H[(size_t)m * ldc + n] = gelu(v);
                }
            }
}

// dZ = dH * gelu'(Z), elementwise.
// (dH and dZ may be the same buffer.)
__global__ void gelu_backward_kernel(size_t n, const float* dH, const float* __restrict__ Z, float* dZ) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dZ[i] = dH[i] * gelu_grad(Z[i]);
}

// out[c] = sum over rows of X[r * cols + c], rows in increasing order (one thread per column).
__global__ void column_sum_kernel(int rows, int cols, const float* __restrict__ X, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < rows; ++r) s += X[(size_t)r * cols + c];
    out[c] = s;
}

// Loss and output gradient of the mean squared error in standardised target
// space: t_std = (t - y_mean)/y_std, loss = mean((y - t_std)^2),
// dY = 2 (y - t_std)/(rows * cols).  One block; fixed-order reduction.
__global__ void mse_kernel(int rows, int cols, const float* __restrict__ Y, const float* __restrict__ T,
                           const float* __restrict__ y_mean, const float* __restrict__ y_inv_std,
                           float* __restrict__ dY, float* __restrict__ loss_out) {
    __shared__ double part[256];
    const size_t n = (size_t)rows * cols;
    double acc = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int c = (int)(i % cols);
        const float ts = (T[i] - y_mean[c]) * y_inv_std[c];
        const float d = Y[i] - ts;
        dY[i] = 2.0f * d / (float)n;
        acc += (double)d * (double)d;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss_out) *loss_out = (float)(part[0] / (double)n);
}

// Adam (Kingma & Ba) with bias correction; the step counter lives on the device.
__global__ void adam_kernel(size_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, const int* __restrict__ step, float lr, float b1, float b2,
                            float eps) {
    const int t = *step + 1;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void step_increment_kernel(int* step, const float* loss, float* loss_hist) {
    if (loss_hist) loss_hist[*step] = *loss;
    *step += 1;
}

// Output de-standardisation: Y = Y * y_std + y_mean.
__global__ void unscale_kernel(size_t n, int cols, float* __restrict__ Y, const float* __restrict__ y_mean,
                               const float* __restrict__ y_std) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % cols);
        Y[i] = Y[i] * y_std[c] + y_mean[c];
    }
}

// Column mean and standard deviation (M-1 denominator) in FP64, fixed order.
__global__ void column_moments_kernel(int rows, int cols, const float* __restrict__ X, double* __restrict__ mean,
                                      double* __restrict__ sdev) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += (double)X[(size_t)r * cols + c];
    const double mu = s / rows;
    double q = 0.0;
    for (int r = 0; r < rows; ++r) {
        const double d = (double)X[(size_t)r * cols + c] - mu;
        q += d * d;
    }
    mean[c] = mu;
    sdev[c] = rows > 1 ? sqrt(q / (rows - 1)) : 0.0;
}

// Features of one cloud per block: bubbles ordered by the gap between the
// bubble's surface and the domain centre, |x_b - c| - r_b (ties by bubble
// index), each as ((x - c)/s, (y - c)/s, (z - c)/s, r/s).
__global__ void features_kernel(int n_clouds, int nb, int keep, const double* __restrict__ bub, double centre,
                                double inv_scale, float* __restrict__ X) {
    extern __shared__ double skey[];
    const int cl = blockIdx.x;
    if (cl >= n_clouds) return;
    const double* b = bub + (size_t)cl * nb * 4;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const double dx = b[4 * i] - centre, dy = b[4 * i + 1] - centre, dz = b[4 * i + 2] - centre;
        skey[i] = sqrt(dx * dx + dy * dy + dz * dz) - b[4 * i + 3];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const double ki = skey[i];
        int rank = 0;
        for (int j = 0; j < nb; ++j) rank += (skey[j] < ki || (skey[j] == ki && j < i)) ? 1 : 0;
        if (rank >= keep) continue;
        float* o = X + (size_t)cl * keep * 4 + 4 * rank;
        o[0] = (float)((b[4 * i] - centre) * inv_scale);
        o[1] = (float)((b[4 * i + 1] - centre) * inv_scale);
        o[2] = (float)((b[4 * i + 2] - centre) * inv_scale);
        o[3] = (float)(b[4 * i + 3] * inv_scale);
    }
}

#define MLP_TRY(call)                                                                      \
    do {                                                                                   \
        cudaError_t err__ = (call);                                                        \
        if (err__ != cudaSuccess)                                                          \
            return fail(OFM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(err__));     \
    } while (0)

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct ofm_mlp {
    int d_in, hidden, n_hidden, d_out, max_rows, n_layers;
    int fan_in[OFM_MLP_MAX_LAYERS], fan_out[OFM_MLP_MAX_LAYERS];
    size_t w_off[OFM_MLP_MAX_LAYERS], b_off[OFM_MLP_MAX_LAYERS];  // offsets in floats within params
    size_t n_params;
    unsigned char* ws;
    bool own_ws;
    float *params, *grads, *m, *v;
    float *Z[OFM_MLP_MAX_LAYERS], *H[OFM_MLP_MAX_LAYERS];  // per layer, max_rows x fan_out
    float *dA, *dB;      // max_rows x max width
    float *x_mean, *x_inv_std, *y_mean, *y_std, *y_inv_std;
    float* loss;
    int* step;
    float* loss_hist;    // OFM_MLP_MAX_STEPS
    cudaGraphExec_t train_graph;
    bool graph_ready;
    const float* graph_X;
    const float* graph_T;
    int graph_n;
    float graph_lr;
};

namespace {

int layout_mlp(ofm_mlp* p, size_t* total) {
    size_t at = 0;
    auto take = [&](size_t bytes) {
        const size_t o = at;
        at = a256(at + bytes);
        return o;
    };
    p->n_layers = p->n_hidden + 1;
    size_t np = 0;
    int maxw = p->d_in;
    for (int l = 0; l < p->n_layers; ++l) {
        p->fan_in[l] = l == 0 ? p->d_in : p->hidden;
        p->fan_out[l] = l == p->n_layers - 1 ? p->d_out : p->hidden;
        p->w_off[l] = np;
        np += (size_t)p->fan_in[l] * p->fan_out[l];
        p->b_off[l] = np;
        np += p->fan_out[l];
        if (p->fan_out[l] > maxw) maxw = p->fan_out[l];
    }
    p->n_params = np;
    size_t o_params = take(np * 4), o_grads = take(np * 4), o_m = take(np * 4), o_v = take(np * 4);
    size_t o_Z[OFM_MLP_MAX_LAYERS], o_H[OFM_MLP_MAX_LAYERS];
    for (int l = 0; l < p->n_layers; ++l) {
        o_Z[l] = take((size_t)p->max_rows * p->fan_out[l] * 4);
        o_H[l] = take((size_t)p->max_rows * p->fan_out[l] * 4);
    }
    size_t o_dA = take((size_t)p->max_rows * maxw * 4), o_dB = take((size_t)p->max_rows * maxw * 4);
    size_t o_xm = take(p->d_in * 4), o_xs = take(p->d_in * 4);
    size_t o_ym = take(p->d_out * 4), o_ys = take(p->d_out * 4), o_yi = take(p->d_out * 4);
    size_t o_loss = take(16), o_step = take(16), o_hist = take(OFM_MLP_MAX_STEPS * 4);
    *total = at;
    if (p->ws) {
        unsigned char* w = p->ws;
        p->params = (float*)(w + o_params);
        p->grads = (float*)(w + o_grads);
        p->m = (float*)(w + o_m);
        p->v = (float*)(w + o_v);
        for (int l = 0; l < p->n_layers; ++l) {
            p->Z[l] = (float*)(w + o_Z[l]);
            p->H[l] = (float*)(w + o_H[l]);
        }
        p->dA = (float*)(w + o_dA);
        p->dB = (float*)(w + o_dB);
        p->x_mean = (float*)(w + o_xm);
        p->x_inv_std = (float*)(w + o_xs);
        p->y_mean = (float*)(w + o_ym);
        p->y_std = (float*)(w + o_ys);
        p->y_inv_std = (float*)(w + o_yi);
        p->loss = (float*)(w + o_loss);
        p->step = (int*)(w + o_step);
        p->loss_hist = (float*)(w + o_hist);
    }
    return OFM_OK;
}

template <bool TA, bool TB>
int gemm(cudaStream_t st, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
         const float* bias, int epi, float* H, const float* shift, const float* scale) {
    const dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
    gemm_kernel<TA, TB><<<grid, GTHREADS, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, epi, H, shift, scale);
    MLP_TRY(cudaGetLastError());
    return OFM_OK;
}

// Forward pass of rows [0, n) of X (n <= max_rows) into the layer buffers;
// the output layer's standardised prediction is Z[L-1].
int forward_rows(ofm_mlp* p, const float* X, int n, cudaStream_t st) {
    const float* in = X;
    for (int l = 0; l < p->n_layers; ++l) {
        const bool last = l == p->n_layers - 1;
        int rc = gemm<false, false>(st, n, p->fan_out[l], p->fan_in[l], in, p->fan_in[l], p->params + p->w_off[l],
                                    p->fan_out[l], p->Z[l], p->fan_out[l], p->params + p->b_off[l],
                                    last ? EPI_BIAS : EPI_BIAS_GELU, p->H[l], l == 0 ? p->x_mean : nullptr,
                                    l == 0 ? p->x_inv_std : nullptr);
        if (rc != OFM_OK) return rc;
        in = p->H[l];
    }
    return OFM_OK;
}

// Loss, backward pass and gradients for rows [0, n) (after forward_rows).
int backward_rows(ofm_mlp* p, const float* X, const float* T, int n, cudaStream_t st) {
    const int L = p->n_layers;
    mse_kernel<<<1, 256, 0, st>>>(n, p->d_out, p->Z[L - 1], T, p->y_mean, p->y_inv_std, p->dA, p->loss);
    MLP_TRY(cudaGetLastError());
    float* dZ = p->dA;  // gradient w.r.t. the current layer's pre-activation
    float* dH = p->dB;
    for (int l = L - 1; l >= 0; --l) {
        const float* in = l == 0 ? X : p->H[l - 1];
        // dW_l = in^T dZ  (fan_in x fan_out)
        int rc = gemm<true, false>(st, p->fan_in[l], p->fan_out[l], n, in, p->fan_in[l], dZ, p->fan_out[l],
                                   p->grads + p->w_off[l], p->fan_out[l], nullptr, EPI_STORE, nullptr,
                                   l == 0 ? p->x_mean : nullptr, l == 0 ? p->x_inv_std : nullptr);
        if (rc != OFM_OK) return rc;
        column_sum_kernel<<<(p->fan_out[l] + 127) / 128, 128, 0, st>>>(n, p->fan_out[l], dZ, p->grads + p->b_off[l]);
        MLP_TRY(cudaGetLastError());
        if (l == 0) break;
        // dH_{l-1} = dZ W_l^T  (n x fan_in)
        rc = gemm<false, true>(st, n, p->fan_in[l], p->fan_out[l], dZ, p->fan_out[l], p->params + p->w_off[l],
                               p->fan_out[l], dH, p->fan_in[l], nullptr, EPI_STORE, nullptr, nullptr, nullptr);
        if (rc != OFM_OK) return rc;
        const size_t cnt = (size_t)n * p->fan_in[l];
        gelu_backward_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, dH, p->Z[l - 1], dH);
        MLP_TRY(cudaGetLastError());
        float* tmp = dZ;
        dZ = dH;
        dH = tmp;
    }
    return OFM_OK;
}

int train_step(ofm_mlp* p, const float* X, const float* T, int n, float lr, cudaStream_t st) {
    int rc = forward_rows(p, X, n, st);
    if (rc != OFM_OK) return rc;
    rc = backward_rows(p, X, T, n, st);
    if (rc != OFM_OK) return rc;
    const unsigned blocks = (unsigned)std::min<size_t>((p->n_params + 255) / 256, 4096);
    adam_kernel<<<blocks, 256, 0, st>>>(p->n_params, p->params, p->grads, p->m, p->v, p->step, lr, 0.9f, 0.999f, 1e-8f);
    MLP_TRY(cudaGetLastError());
    step_increment_kernel<<<1, 1, 0, st>>>(p->step, p->loss, p->loss_hist);
    MLP_TRY(cudaGetLastError());
    return OFM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int ofm_mlp_workspace_bytes(int d_in, int hidden, int n_hidden, int d_out, int max_rows, size_t* bytes) {
    ofm::clear_error();
    if (d_in < 1 || hidden < 1 || n_hidden < 1 || n_hidden + 1 > OFM_MLP_MAX_LAYERS || d_out < 1 || max_rows < 1 ||
        !bytes)
        return fail(OFM_EINVAL, "ofm_mlp_workspace_bytes: bad sizes");
    // a weight matrix or an activation array of more than 2^40 values would not
    // fit any device; bounding them keeps every byte count below 2^50 (no wrap)
    const long long wmax = std::max<long long>({(long long)d_in, (long long)hidden, (long long)d_out});
    if ((long long)d_in * hidden > (1LL << 40) || (long long)hidden * hidden > (1LL << 40) ||
        (long long)hidden * d_out > (1LL << 40) || (long long)max_rows * wmax > (1LL << 40))
        return fail(OFM_ENOMEM, "ofm_mlp_workspace_bytes: network too large (%d inputs, %d wide, %d outputs, %d rows)",
                    d_in, hidden, d_out, max_rows);
    ofm_mlp p;
    std::memset(&p, 0, sizeof(p));
    p.d_in = d_in;
    p.hidden = hidden;
    p.n_hidden = n_hidden;
    p.d_out = d_out;
    p.max_rows = max_rows;
    return layout_mlp(&p, bytes);
}

extern "C" int ofm_mlp_create(ofm_mlp** out, int d_in, int hidden, int n_hidden, int d_out, int max_rows,
                              void* workspace, size_t workspace_bytes) {
    ofm::clear_error();
    if (!out) return fail(OFM_EINVAL, "ofm_mlp_create: NULL out");
    *out = nullptr;
    size_t need = 0;
    int rc = ofm_mlp_workspace_bytes(d_in, hidden, n_hidden, d_out, max_rows, &need);
    if (rc != OFM_OK) return rc;
    if (((uintptr_t)workspace) % 256 != 0) return fail(OFM_EINVAL, "workspace must be 256-byte aligned");
    ofm_mlp* p = new (std::nothrow) ofm_mlp;
    if (!p) return fail(OFM_ENOMEM, "out of host memory");
    std::memset(p, 0, sizeof(*p));
    p->d_in = d_in;
    p->hidden = hidden;
    p->n_hidden = n_hidden;
    p->d_out = d_out;
    p->max_rows = max_rows;
    if (workspace) {
        if (workspace_bytes < need) {
            delete p;
            return fail(OFM_ENOMEM, "workspace has %zu bytes, the network needs %zu", workspace_bytes, need);
        }
        p->ws = (unsigned char*)workspace;
    } else {
        if (cudaMalloc((void**)&p->ws, need) != cudaSuccess) {
            delete p;
            return fail(OFM_ENOMEM, "cudaMalloc(%zu) failed", need);
        }
        p->own_ws = true;
    }
    layout_mlp(p, &need);
    if (cudaMemset(p->ws, 0, need) != cudaSuccess) {
        ofm_mlp_destroy(p);
        return fail(OFM_ECUDA, "cudaMemset failed");
    }
    // identity scaling until the caller sets one
    std::vector<float> ones(std::max(d_in, d_out), 1.0f);
    if (cudaMemcpy(p->x_inv_std, ones.data(), d_in * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->y_std, ones.data(), d_out * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->y_inv_std, ones.data(), d_out * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        ofm_mlp_destroy(p);
        return fail(OFM_ECUDA, "scaling upload failed");
    }
    *out = p;
    return OFM_OK;
}

extern "C" void ofm_mlp_destroy(ofm_mlp* p) {
    if (!p) return;
    if (p->graph_ready) cudaGraphExecDestroy(p->train_graph);
    if (p->own_ws && p->ws) cudaFree(p->ws);
    delete p;
}

extern "C" int ofm_mlp_param_count(const ofm_mlp* p, int64_t* n) {
    if (!p || !n) return fail(OFM_EINVAL, "NULL argument");
    *n = (int64_t)p->n_params;
    return OFM_OK;
}

extern "C" int ofm_mlp_set_params(ofm_mlp* p, const float* host) {
    ofm::clear_error();
    if (!p || !host) return fail(OFM_EINVAL, "NULL argument");
    MLP_TRY(cudaMemcpy(p->params, host, p->n_params * 4, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemset(p->m, 0, p->n_params * 4));
    MLP_TRY(cudaMemset(p->v, 0, p->n_params * 4));
    MLP_TRY(cudaMemset(p->step, 0, sizeof(int)));
    return OFM_OK;
}

extern "C" int ofm_mlp_get_params(ofm_mlp* p, float* host) {
    ofm::clear_error();
    if (!p || !host) return fail(OFM_EINVAL, "NULL argument");
    MLP_TRY(cudaMemcpy(host, p->params, p->n_params * 4, cudaMemcpyDeviceToHost));
    return OFM_OK;
}

extern "C" int ofm_mlp_set_scaling(ofm_mlp* p, const float* x_mean, const float* x_std, const float* y_mean,
                                   const float* y_std) {
    ofm::clear_error();
    if (!p || !x_mean || !x_std || !y_mean || !y_std) return fail(OFM_EINVAL, "NULL argument");
    std::vector<float> xi(p->d_in), yi(p->d_out);
    for (int i = 0; i < p->d_in; ++i) xi[i] = x_std[i] > 0.0f ? 1.0f / x_std[i] : 1.0f;
    for (int i = 0; i < p->d_out; ++i) yi[i] = y_std[i] > 0.0f ? 1.0f / y_std[i] : 1.0f;
    MLP_TRY(cudaMemcpy(p->x_mean, x_mean, p->d_in * 4, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(p->x_inv_std, xi.data(), p->d_in * 4, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(p->y_mean, y_mean, p->d_out * 4, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(p->y_std, y_std, p->d_out * 4, cudaMemcpyHostToDevice));
    MLP_TRY(cudaMemcpy(p->y_inv_std, yi.data(), p->d_out * 4, cudaMemcpyHostToDevice));
    return OFM_OK;
}

extern "C" int ofm_mlp_forward(ofm_mlp* p, const float* X, int n, float* Y, void* stream) {
    ofm::clear_error();
    if (!p || !X || !Y || n < 0) return fail(OFM_EINVAL, "ofm_mlp_forward: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int L = p->n_layers;
    for (int r0 = 0; r0 < n; r0 += p->max_rows) {
        const int rows = std::min(p->max_rows, n - r0);
        int rc = forward_rows(p, X + (size_t)r0 * p->d_in, rows, st);
        if (rc != OFM_OK) return rc;
        MLP_TRY(cudaMemcpyAsync(Y + (size_t)r0 * p->d_out, p->Z[L - 1], (size_t)rows * p->d_out * 4,
                                cudaMemcpyDeviceToDevice, st));
        const size_t cnt = (size_t)rows * p->d_out;
        unscale_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, p->d_out, Y + (size_t)r0 * p->d_out,
                                                                       p->y_mean, p->y_std);
        MLP_TRY(cudaGetLastError());
    }
    return OFM_OK;
}

extern "C" int ofm_mlp_gradients(ofm_mlp* p, const float* X, const float* T, int n, float* grads_host,
                                 float* loss_host, void* stream) {
    ofm::clear_error();
    if (!p || !X || !T || n < 1 || n > p->max_rows) return fail(OFM_EINVAL, "ofm_mlp_gradients: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = forward_rows(p, X, n, st);
    if (rc != OFM_OK) return rc;
    rc = backward_rows(p, X, T, n, st);
    if (rc != OFM_OK) return rc;
    if (grads_host) MLP_TRY(cudaMemcpyAsync(grads_host, p->grads, p->n_params * 4, cudaMemcpyDeviceToHost, st));
    if (loss_host) MLP_TRY(cudaMemcpyAsync(loss_host, p->loss, 4, cudaMemcpyDeviceToHost, st));
    MLP_TRY(cudaStreamSynchronize(st));
    return OFM_OK;
}

extern "C" int ofm_mlp_train(ofm_mlp* p, const float* X, const float* T, int n, int steps, float lr,
                             float* loss_hist_host, void* stream) {
    ofm::clear_error();
    if (!p || !X || !T || n < 1 || n > p->max_rows || steps < 0 || !(lr > 0.0f))
        return fail(OFM_EINVAL, "ofm_mlp_train: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    int step0 = 0;
    MLP_TRY(cudaMemcpyAsync(&step0, p->step, sizeof(int), cudaMemcpyDeviceToHost, st));
    MLP_TRY(cudaStreamSynchronize(st));
    if (step0 + steps > OFM_MLP_MAX_STEPS) return fail(OFM_EINVAL, "ofm_mlp_train: more than %d steps", OFM_MLP_MAX_STEPS);
    // one training step captured once per (X, T, n, lr) and replayed
    if (!p->graph_ready || p->graph_X != X || p->graph_T != T || p->graph_n != n || p->graph_lr != lr) {
        if (p->graph_ready) {
            cudaGraphExecDestroy(p->train_graph);
            p->graph_ready = false;
        }
        cudaStream_t cap;
        MLP_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaStreamDestroy(cap);
            return fail(OFM_ECUDA, "begin capture failed");
        }
        int rc = train_step(p, X, T, n, lr, cap);
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (rc != OFM_OK) return rc;
        if (e != cudaSuccess) return fail(OFM_ECUDA, "end capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&p->train_graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(OFM_ECUDA, "instantiate: %s", cudaGetErrorString(e));
        p->graph_ready = true;
        p->graph_X = X;
        p->graph_T = T;
        p->graph_n = n;
        p->graph_lr = lr;
    }
    for (int s = 0; s < steps; ++s) MLP_TRY(cudaGraphLaunch(p->train_graph, st));
    if (loss_hist_host && steps > 0)
        MLP_TRY(cudaMemcpyAsync(loss_hist_host, p->loss_hist + step0, steps * 4, cudaMemcpyDeviceToHost, st));
    MLP_TRY(cudaStreamSynchronize(st));
    return OFM_OK;
}

extern "C" int ofm_column_moments(const float* X, int rows, int cols, double* mean_dev, double* std_dev, void* stream) {
    ofm::clear_error();
    if (!X || rows < 1 || cols < 1 || !mean_dev || !std_dev) return fail(OFM_EINVAL, "ofm_column_moments: bad arguments");
    column_moments_kernel<<<(cols + 127) / 128, 128, 0, (cudaStream_t)stream>>>(rows, cols, X, mean_dev, std_dev);
    MLP_TRY(cudaGetLastError());
    return OFM_OK;
}

extern "C" int ofm_cloud_features(const double* bubbles_dev, int n_clouds, int n_bubbles, int n_keep,
                                  double domain_L, double scale, float* X_dev, void* stream) {
    ofm::clear_error();
    if (!bubbles_dev || !X_dev || n_clouds < 0 || n_bubbles < 1 || n_bubbles > 4096 || !(scale > 0.0) ||
        n_keep < 0 || n_keep > n_bubbles)
        return fail(OFM_EINVAL, "ofm_cloud_features: bad arguments");
    if (n_clouds == 0) return OFM_OK;
    const int keep = n_keep == 0 ? n_bubbles : n_keep;
    const size_t sm = (size_t)n_bubbles * sizeof(double);
    features_kernel<<<n_clouds, 128, sm, (cudaStream_t)stream>>>(n_clouds, n_bubbles, keep, bubbles_dev,
                                                                 0.5 * domain_L, 1.0 / scale, X_dev);
    MLP_TRY(cudaGetLastError());
    return OFM_OK;
}
