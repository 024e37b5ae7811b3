// sketch.cu -- planner features of a join instance (K12) and the cost model.
//
// Features (24 floats, the input of the learned planner):
//   0-2   log2(1 + |R|), log2(1 + |S|), log2(1 + |T|)
//   3-6   log2(1 + distinct values) of R.x, R.y, S.y, T.y (HyperLogLog)
//   7     1 for the cyclic join, 0 for the linear one
//   8     log2(1 + estimated |R join S|): m sampled S tuples, the exact
//         number of R tuples sharing each sampled B value, scaled by |S|/m
//         (an unbiased estimate of sum_b deg_R(b) deg_S(b), the cascade's
//         intermediate size and the cyclic join's wedge count)
//   9-23  sampled key-frequency profile: for R.y, S.x, S.y, T.x and (cyclic)
//         T.y, the fractions of m sampled keys whose value occurs once, 2-7
//         times and 8+ times in the sample (5 columns x 3 bins)
//
// The cost model (Appendix A restated for this GPU: a plan's time is the
// sum of its phases, each the larger of its bytes over HBM bandwidth and its
// random lookups over the L2 lookup rate) predicts both plans' times from
// the same features and is the planner's fallback.
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <vector>

#include "api_internal.h"
#include "prof.h"
#include "tables.h"

namespace mwj {
namespace {

constexpr int ST = 512;
constexpr uint32_t kSample = 4096;
constexpr uint32_t kSampleSlots = 8192;

__global__ void k_gather_stride(const int32_t *__restrict__ col, uint32_t n, uint32_t m,
                                int32_t *__restrict__ out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const uint64_t src = (uint64_t)i * n / m;   // evenly spaced sample positions
        out[i] = __ldg(col + src);
    }
}

// deg[k] = occurrences in col of the k-th distinct sampled key (keys given)
__global__ void __launch_bounds__(ST) k_sample_degrees(const int32_t *__restrict__ col, uint32_t n,
                                                       const int32_t *__restrict__ keys, uint32_t nk,
                                                       uint32_t seed,
                                                       unsigned long long *__restrict__ deg) {
    __shared__ uint32_t tk[kSampleSlots + 1];
    __shared__ uint32_t tc[kSampleSlots + 1];
    __shared__ int32_t slot_at[kSample];
    const uint32_t mask = kSampleSlots - 1;
    for (uint32_t s = threadIdx.x; s <= kSampleSlots; s += ST) {
        tk[s] = (s < kSampleSlots) ? kEmptyKey : 0u;
        tc[s] = 0u;
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < nk; k += ST) {
        bool fresh;
        slot_at[k] = tbl_insert(tk, mask, (uint32_t)keys[k], seed, &fresh);
    }
    __syncthreads();
    for (uint32_t i = blockIdx.x * ST + threadIdx.x; i < n; i += gridDim.x * ST) {
        int s = tbl_find(tk, mask, (uint32_t)__ldg(col + i), seed);
        if (s >= 0) atomicAdd(&tc[s], 1u);
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < nk; k += ST) {
        int s = slot_at[k];
        if (s >= 0 && tc[s]) {
            // every sampled key k receives its slot's count once per CTA
            atomicAdd(deg + k, (unsigned long long)tc[s]);
        }
    }
}

uint32_t hll_estimate(const std::vector<unsigned int> &regs) {
    const double m = (double)regs.size();
    double S = 0.0;
    unsigned z = 0;
    for (unsigned r : regs) {
        S += std::ldexp(1.0, -(int)r);
        z += (r == 0);
    }
    double E = (0.7213 / (1.0 + 1.079 / m)) * m * m / S;
    if (E <= 2.5 * m && z > 0) E = m * std::log(m / (double)z);
    return (uint32_t)std::min(E, 4294967295.0);
}

}  // namespace

size_t sketch_workspace_bytes() {
    return align256(hll_scratch_registers(256) * 4 + 16) + align256(kSample * 4 + 16) +
           align256(kSample * 8 + 16);
}

mwj_status compute_features(mwj_ctx *ctx, int kind, const mwj_rel &R, const mwj_rel &S,
                            const mwj_rel &T, void *ws, size_t ws_bytes, cudaStream_t st, float *f) {
    if (ws_bytes < sketch_workspace_bytes() || !ws) return fail(ctx, MWJ_ERR_WORKSPACE, "sketch workspace");
    unsigned int *regs = (unsigned int *)ws;
    if (ctx->dev.num_sms > 256) return fail(ctx, MWJ_ERR_UNIMPLEMENTED, "more than 256 SMs");
    int32_t *samp = (int32_t *)((char *)ws + align256(hll_scratch_registers(256) * 4 + 16));
    unsigned long long *deg =
        (unsigned long long *)((char *)samp + align256(kSample * 4 + 16));
    const int sms = ctx->dev.num_sms;
    cudaError_t e;
    auto hll_of = [&](const int32_t *col, int64_t n) -> double {
        if (n <= 0) return 0.0;
        e = hll_regs(col, n, ctx->seeds.D, regs, sms, st);
        std::vector<unsigned int> h(hll_registers());
        cudaMemcpyAsync(h.data(), regs, h.size() * 4, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        return (double)hll_estimate(h);
    };
    auto sample_of = [&](const int32_t *col, int64_t n, std::vector<int32_t> &out) {
        out.clear();
        if (n <= 0) return;
        const uint32_t m = (uint32_t)std::min<int64_t>(n, kSample);
        {
            ProfScope ps_("sketch_sample", st);
            k_gather_stride<<<(m + 255) / 256, 256, 0, st>>>(col, (uint32_t)n, m, samp);
        }
        out.resize(m);
        cudaMemcpyAsync(out.data(), samp, m * 4, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
    };
    for (int k = 0; k < 24; ++k) f[k] = 0.f;
    f[0] = (float)std::log2(1.0 + R.n);
    f[1] = (float)std::log2(1.0 + S.n);
    f[2] = (float)std::log2(1.0 + T.n);
    f[3] = (float)std::log2(1.0 + hll_of(R.x, R.n));
    f[4] = (float)std::log2(1.0 + hll_of(R.y, R.n));
    f[5] = (float)std::log2(1.0 + hll_of(S.y, S.n));
    f[6] = (float)std::log2(1.0 + hll_of(T.y, T.n));
    f[7] = kind == MWJ_CYCLIC ? 1.f : 0.f;
    // |R join S| from sampled S tuples' exact degrees in R
    std::vector<int32_t> sb;
    sample_of(S.x, S.n, sb);
    double inter = 0.0;
    if (!sb.empty() && R.n > 0) {
        const uint32_t m = (uint32_t)sb.size();
        cudaMemcpyAsync(samp, sb.data(), m * 4, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(deg, 0, m * 8, st);
        {
            ProfScope ps_("sketch_degrees", st);
            const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(sms * 2, (R.n + 65535) / 65536));
            k_sample_degrees<<<grid, ST, 0, st>>>(R.y, (uint32_t)R.n, samp, m, ctx->seeds.slot, deg);
        }
        std::vector<unsigned long long> d(m);
        cudaMemcpyAsync(d.data(), deg, m * 8, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        double s = 0.0;
        for (uint32_t k = 0; k < m; ++k) s += (double)d[k];
        inter = s * (double)S.n / (double)m;
    }
    f[8] = (float)std::log2(1.0 + inter);
    // sampled key-frequency profiles
    const int32_t *cols[5] = {R.y, S.x, S.y, T.x, kind == MWJ_CYCLIC ? T.y : nullptr};
    const int64_t ns[5] = {R.n, S.n, S.n, T.n, T.n};
    for (int c = 0; c < 5; ++c) {
        if (!cols[c]) continue;
        std::vector<int32_t> smp;
        sample_of(cols[c], ns[c], smp);
        if (smp.empty()) continue;
        std::unordered_map<int32_t, uint32_t> cnt;
        for (int32_t v : smp) cnt[v]++;
        double b0 = 0, b1 = 0, b2 = 0;
        for (int32_t v : smp) {
            uint32_t q = cnt[v];
            if (q <= 1) b0 += 1; else if (q < 8) b1 += 1; else b2 += 1;
        }
        const double m = (double)smp.size();
        f[9 + 3 * c] = (float)(b0 / m);
        f[10 + 3 * c] = (float)(b1 / m);
        f[11 + 3 * c] = (float)(b2 / m);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "sketch");
    return MWJ_OK;
}

// ---- cost model ------------------------------------------------------------
// log2 predicted seconds of the three plans a planner weighs: out[0] the
// cascade, out[1] the 3-way join with the default shares, out[2] with the
// alternative shares (mwj_plan_shares_alt).  Each phase costs its slowest
// resource (Appendix A): HBM bytes at hbm_gbs, random lookups into an
// L2-resident table, or on-chip wedge probes, plus a fixed cost per call.
// The byte counts restate the paper's tuple counts:
//   linear 3-way join (Section 4.2): R and S read once, T held whole (the
//     |R||T|/M term vanishes while T's table fits on chip);
//   cascade (Example 3, Section 6.3): R join S written as I and read back,
//     12 bytes per I row each way, one T lookup per I row (the cyclic
//     cascade writes I once more, grouped by (c, a), 8 bytes per row);
//   cyclic cube tiling (Section 5.2): |R| + 2 sqrt(|R||S||T|/M) tuples read
//     at the optimal share, M the tuples of one on-chip tile, and every wedge
//     of R join S checked once on chip.
void cost_model(const float *f, double hbm_gbs, double *out) {
    const double nR = std::exp2(f[0]) - 1, nS = std::exp2(f[1]) - 1, nT = std::exp2(f[2]) - 1;
    const double dB = std::exp2(f[4]) - 1, dC = std::exp2(f[5]) - 1;   // distinct B (of R), C (of S)
    const double nI = std::exp2(f[8]) - 1;        // |R join S| estimate
    const bool cyc = f[7] > 0.5f;
    const double bw = hbm_gbs * 1e9;              // bytes/s
    const double call = 40e-6;                    // launches and host work of one call
    const double l2_table = 64e6;                 // bytes of a lookup table the L2 keeps
    // random lookups/s into a table of `keys` distinct keys (8-byte slots at
    // most a quarter full): L2-resident, else served by HBM sectors
    auto lookups = [&](double keys) { return 32.0 * keys <= l2_table ? 2.6e11 : 1.0e11; };
    const double wedge_c = 2.3e11;                // C-bucket probe: wedge checks/s
    const double wedge_t = 1.5e10;                // cube tiles: wedge checks/s
    const double M = 1024.0;                      // tuples of R (and of T) one cube tile holds
    const double tile = 8e-6 / 304.0;             // rebuilding one cube tile, spread over the CTAs
    double tc, tm, ta;
    if (!cyc) {
        const double Lb = lookups(std::max(dB, 1.0)), Lc = lookups(std::max(dC, 1.0));
        const double passes = std::max(8.0 * (nR + nS) / bw, nS / Lc + nR / Lb);
        tm = call + 12.0 * nT / bw + passes;                          // one bucket per side
        ta = call + 16.0 * (nR + nS) / bw + 12.0 * nT / bw + passes;  // + partitioning R and S
        tc = 2 * call + 16.0 * (nR + nS) / bw + 12.0 * nT / bw + 12.0 * nI / bw +
             std::max(12.0 * nI / bw, nI / Lc);
    } else {
        const double Lb = lookups(std::max(dB, 1.0));
        tm = call + 16.0 * nR / bw + nR / Lb + 20.0 * (nS + nT) / bw + nS / Lb + nI / wedge_c;
        const double reads = nR + 2.0 * std::sqrt(std::max(1.0, nR * nS * nT / M));
        const double H = std::max(1.0, std::sqrt(nR * nT / (M * std::max(nS, 1.0))));
        const double tiles = std::max(1.0, nR / M) * H;
        ta = call + 20.0 * (nR + nS + nT) / bw + 8.0 * reads / bw + tiles * tile + nI / wedge_t;
        tc = 2 * call + 16.0 * (nR + nS) / bw + 12.0 * nI / bw + 20.0 * (nI + nT) / bw + nI / Lb;
    }
    out[0] = std::log2(std::max(tc, 1e-7));
    out[1] = std::log2(std::max(tm, 1e-7));
    out[2] = std::log2(std::max(ta, 1e-7));
}

}  // namespace mwj

using namespace mwj;

extern "C" {

mwj_status mwj_features(mwj_ctx *ctx, int kind, mwj_rel R, mwj_rel S, mwj_rel T, float *features,
                        void *workspace, size_t ws_bytes, void *stream) {
    if (!ctx || !features) return MWJ_ERR_INVALID_ARG;
    if (kind != MWJ_LINEAR && kind != MWJ_CYCLIC) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad kind");
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    ApiScope api_scope(&ctx->prof);
    return compute_features(ctx, kind, R, S, T, workspace, ws_bytes, (cudaStream_t)stream, features);
}

size_t mwj_features_workspace_size(void) { return sketch_workspace_bytes(); }

mwj_status mwj_cost_model(const float *features, double hbm_gbs, double *out3) {
    if (!features || !out3 || hbm_gbs <= 0) return MWJ_ERR_INVALID_ARG;
    cost_model(features, hbm_gbs, out3);
    return MWJ_OK;
}

}  // extern "C"
