// mlp.cu -- the learned planner's network: 24 -> 128 -> 128 -> 3, ReLU.
//
// Weights and activations are BF16 (round to nearest even), every product
// is accumulated in FP32, gradients are FP32, and Adam keeps FP32 master
// weights from which the BF16 copy is refreshed after every step.  At this
// size the layers are a few hundred thousand multiply-adds per row block, so
// plain FMA on BF16-rounded operands is used rather than tensor cores.
//
// Parameter layout (FP32 master and BF16 copy alike): W1[24][128], b1[128],
// W2[128][128], b2[128], W3[128][3], b3[3]; W[k][j] multiplies input k into
// output j.  Loss: sum over rows r and outputs o of M[r][o] (Y[r][o] -
// T[r][o])^2, divided by the number of nonzero M entries.
#include <cuda_bf16.h>

#include "api_internal.h"
#include "prof.h"

namespace mwj {
namespace {

constexpr int NIN = 24, NH = 128, NOUT = 3;
constexpr int OW1 = 0, OB1 = OW1 + NIN * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NOUT, NPARAM = OB3 + NOUT;
constexpr int MT = 128;   // threads per block: one per hidden unit
constexpr int ROWS = 32;  // rows per block

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float w(const __nv_bfloat16 *p, int i) { return __bfloat162float(p[i]); }

struct Act {
    float x[ROWS][NIN];
    float h1[ROWS][NH];
    float h2[ROWS][NH];
    float y[ROWS][NOUT];
};

// forward of rows [r0, r0 + nr) into the shared activations (all BF16-rounded)
__device__ void forward_block(const __nv_bfloat16 *__restrict__ P, const float *__restrict__ X, int r0,
                              int nr, Act &a) {
    const int j = threadIdx.x;
    for (int i = j; i < ROWS * NIN; i += MT) {
        const int r = i / NIN, k = i % NIN;
        a.x[r][k] = (r < nr) ? bf(X[(size_t)(r0 + r) * NIN + k]) : 0.f;
    }
    __syncthreads();
    {
        float wc[NIN];
#pragma unroll
        for (int k = 0; k < NIN; ++k) wc[k] = w(P, OW1 + k * NH + j);
        const float b = w(P, OB1 + j);
        for (int r = 0; r < ROWS; ++r) {
            float s = b;
#pragma unroll
            for (int k = 0; k < NIN; ++k) s = fmaf(a.x[r][k], wc[k], s);
            a.h1[r][j] = bf(fmaxf(s, 0.f));
        }
    }
    __syncthreads();
    {
        float acc[ROWS];
        const float b = w(P, OB2 + j);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) acc[r] = b;
        for (int k = 0; k < NH; ++k) {
            const float wk = w(P, OW2 + k * NH + j);
#pragma unroll
            for (int r = 0; r < ROWS; ++r) acc[r] = fmaf(a.h1[r][k], wk, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < ROWS; ++r) a.h2[r][j] = bf(fmaxf(acc[r], 0.f));
    }
    __syncthreads();
    for (int i = j; i < ROWS * NOUT; i += MT) {
        const int r = i / NOUT, o = i % NOUT;
        float s = w(P, OB3 + o);
        for (int k = 0; k < NH; ++k) s = fmaf(a.h2[r][k], w(P, OW3 + k * NOUT + o), s);
        a.y[r][o] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(MT) k_mlp_fwd(const __nv_bfloat16 *__restrict__ P,
                                                const float *__restrict__ X, int B,
                                                float *__restrict__ Y) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Act &a = *(Act *)smraw;
    for (int r0 = blockIdx.x * ROWS; r0 < B; r0 += gridDim.x * ROWS) {
        const int nr = min(ROWS, B - r0);
        forward_block(P, X, r0, nr, a);
        for (int i = threadIdx.x; i < nr * NOUT; i += MT) Y[(size_t)r0 * NOUT + i] = a.y[i / NOUT][i % NOUT];
        __syncthreads();
    }
}

// Gradients of the masked mean squared error, summed over the block's rows
// and added into G (FP32); loss accumulated into *loss.
__global__ void __launch_bounds__(MT) k_mlp_bwd(const __nv_bfloat16 *__restrict__ P,
                                                const float *__restrict__ X,
                                                const float *__restrict__ Tg,
                                                const float *__restrict__ Mk, int B, float inv_count,
                                                float *__restrict__ G, float *__restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Act &a = *(Act *)smraw;
    __shared__ float dy[ROWS][NOUT];
    __shared__ float dh2[ROWS][NH];
    __shared__ float dh1[ROWS][NH];
    const int j = threadIdx.x;
    for (int r0 = blockIdx.x * ROWS; r0 < B; r0 += gridDim.x * ROWS) {
        const int nr = min(ROWS, B - r0);
        forward_block(P, X, r0, nr, a);
        float lsum = 0.f;
        for (int i = j; i < ROWS * NOUT; i += MT) {
            const int r = i / NOUT, o = i % NOUT;
            float d = 0.f;
            if (r < nr) {
                const size_t g = (size_t)(r0 + r) * NOUT + o;
                const float m = Mk[g];
                const float e = a.y[r][o] - Tg[g];
                d = 2.f * m * e * inv_count;
                lsum += m * e * e * inv_count;
            }
            dy[r][o] = d;
        }
        if (lsum != 0.f) atomicAdd(loss, lsum);
        __syncthreads();
        // layer 3: dW3[k][o], db3[o]; dH2
        for (int i = j; i < NH * NOUT; i += MT) {
            const int k = i / NOUT, o = i % NOUT;
            float s = 0.f;
            for (int r = 0; r < nr; ++r) s = fmaf(a.h2[r][k], dy[r][o], s);
            atomicAdd(G + OW3 + i, s);
        }
        if (j < NOUT) {
            float s = 0.f;
            for (int r = 0; r < nr; ++r) s += dy[r][j];
            atomicAdd(G + OB3 + j, s);
        }
        {
            const float w0 = w(P, OW3 + j * NOUT), w1 = w(P, OW3 + j * NOUT + 1), w2 = w(P, OW3 + j * NOUT + 2);
            for (int r = 0; r < ROWS; ++r) {
                const float g = dy[r][0] * w0 + dy[r][1] * w1 + dy[r][2] * w2;
                dh2[r][j] = (a.h2[r][j] > 0.f) ? g : 0.f;
            }
        }
        __syncthreads();
        // layer 2: dW2[k][j] (thread j owns output column j), db2[j]; dH1
        {
            float sb = 0.f;
            for (int r = 0; r < nr; ++r) sb += dh2[r][j];
            atomicAdd(G + OB2 + j, sb);
            for (int k = 0; k < NH; ++k) {
                float s = 0.f;
                for (int r = 0; r < nr; ++r) s = fmaf(a.h1[r][k], dh2[r][j], s);
                atomicAdd(G + OW2 + k * NH + j, s);
            }
            // dH1[r][j] = sum_q dH2[r][q] W2[j][q]  (thread j owns input unit j)
            float acc[ROWS];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) acc[r] = 0.f;
            for (int q = 0; q < NH; ++q) {
                const float wq = w(P, OW2 + j * NH + q);
#pragma unroll
                for (int r = 0; r < ROWS; ++r) acc[r] = fmaf(dh2[r][q], wq, acc[r]);
            }
#pragma unroll
            for (int r = 0; r < ROWS; ++r) dh1[r][j] = (a.h1[r][j] > 0.f) ? acc[r] : 0.f;
        }
        __syncthreads();
        // layer 1: dW1[k][j], db1[j]
        {
            float sb = 0.f;
            for (int r = 0; r < nr; ++r) sb += dh1[r][j];
            atomicAdd(G + OB1 + j, sb);
            for (int k = 0; k < NIN; ++k) {
                float s = 0.f;
                for (int r = 0; r < nr; ++r) s = fmaf(a.x[r][k], dh1[r][j], s);
                atomicAdd(G + OW1 + k * NH + j, s);
            }
        }
        __syncthreads();
    }
}

// Adam (Kingma and Ba) on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_mlp_adam(float *__restrict__ P, __nv_bfloat16 *__restrict__ Pb,
                           const float *__restrict__ G, float *__restrict__ m, float *__restrict__ v,
                           float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        const float g = G[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float p = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        P[i] = p;
        Pb[i] = __float2bfloat16_rn(p);
    }
}

__global__ void k_to_bf16(const float *__restrict__ P, __nv_bfloat16 *__restrict__ Pb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x)
        Pb[i] = __float2bfloat16_rn(P[i]);
}

}  // namespace
}  // namespace mwj

using namespace mwj;

struct mwj_mlp {
    mwj_ctx *ctx;
    float *P;             // FP32 master
    __nv_bfloat16 *Pb;    // BF16 copy
    float *m, *v;         // Adam moments
};

extern "C" {

size_t mwj_mlp_num_params(void) { return (size_t)NPARAM; }

mwj_status mwj_mlp_create(mwj_ctx *ctx, mwj_mlp **out) {
    if (!ctx || !out) return MWJ_ERR_INVALID_ARG;
    mwj_mlp *n = new mwj_mlp();
    n->ctx = ctx;
    cudaError_t e = cudaMalloc(&n->P, sizeof(float) * NPARAM * 3 + sizeof(__nv_bfloat16) * NPARAM + 256);
    if (e != cudaSuccess) {
        delete n;
        return cuda_fail(ctx, e, "mlp parameters");
    }
    n->m = n->P + NPARAM;
    n->v = n->m + NPARAM;
    n->Pb = (__nv_bfloat16 *)(n->v + NPARAM);
    cudaMemset(n->P, 0, sizeof(float) * NPARAM * 3 + sizeof(__nv_bfloat16) * NPARAM);
    *out = n;
    return MWJ_OK;
}

mwj_status mwj_mlp_destroy(mwj_mlp *n) {
    if (!n) return MWJ_ERR_INVALID_ARG;
    cudaFree(n->P);
    delete n;
    return MWJ_OK;
}

mwj_status mwj_mlp_set_params(mwj_mlp *n, const float *host) {
    if (!n || !host) return MWJ_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpy(n->P, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(n->ctx, e, "mlp set");
    cudaMemset(n->m, 0, sizeof(float) * NPARAM * 2);
    k_to_bf16<<<(NPARAM + 255) / 256, 256>>>(n->P, n->Pb);
    e = cudaDeviceSynchronize();
    return e == cudaSuccess ? MWJ_OK : cuda_fail(n->ctx, e, "mlp set");
}

mwj_status mwj_mlp_get_params(mwj_mlp *n, float *host) {
    if (!n || !host) return MWJ_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpy(host, n->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MWJ_OK : cuda_fail(n->ctx, e, "mlp get");
}

mwj_status mwj_mlp_forward(mwj_mlp *n, const float *X, int32_t B, float *Y, void *stream) {
    if (!n || B < 0 || (B > 0 && (!X || !Y))) return MWJ_ERR_INVALID_ARG;
    if (B == 0) return MWJ_OK;
    ApiScope api_scope(&n->ctx->prof);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t smem = sizeof(Act);
    cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int blocks = (B + ROWS - 1) / ROWS;
    {
        ProfScope ps_("mlp_forward", st);
        k_mlp_fwd<<<blocks < 1024 ? blocks : 1024, MT, smem, st>>>(n->Pb, X, B, Y);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MWJ_OK : cuda_fail(n->ctx, e, "mlp forward");
}

mwj_status mwj_mlp_backward(mwj_mlp *n, const float *X, const float *T, const float *M, int32_t B,
                            float inv_count, float *grads, float *loss, void *stream) {
    if (!n || B < 0 || !grads || !loss || (B > 0 && (!X || !T || !M))) return MWJ_ERR_INVALID_ARG;
    ApiScope api_scope(&n->ctx->prof);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(grads, 0, sizeof(float) * NPARAM, st)) != cudaSuccess) return cuda_fail(n->ctx, e, "mlp");
    if ((e = cudaMemsetAsync(loss, 0, sizeof(float), st)) != cudaSuccess) return cuda_fail(n->ctx, e, "mlp");
    if (B == 0) return MWJ_OK;
    const size_t smem = sizeof(Act);
    cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int blocks = (B + ROWS - 1) / ROWS;
    {
        ProfScope ps_("mlp_backward", st);
        k_mlp_bwd<<<blocks < 512 ? blocks : 512, MT, smem, st>>>(n->Pb, X, T, M, B, inv_count, grads, loss);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? MWJ_OK : cuda_fail(n->ctx, e, "mlp backward");
}

mwj_status mwj_mlp_adam(mwj_mlp *n, const float *grads, float lr, int32_t step, void *stream) {
    if (!n || !grads || step < 1) return MWJ_ERR_INVALID_ARG;
    ApiScope api_scope(&n->ctx->prof);
    cudaStream_t st = (cudaStream_t)stream;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    {
        ProfScope ps_("mlp_adam", st);
        k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(n->P, n->Pb, grads, n->m, n->v, lr, b1, b2,
                                                          1e-8f, c1, c2);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MWJ_OK : cuda_fail(n->ctx, e, "mlp adam");
}

}  // extern "C"
