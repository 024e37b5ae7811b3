// api_cyclic.cu -- C ABI of the cyclic join: share choice, workspace layout,
// kernel order.
#include <cmath>

#include "api_internal.h"
#include "cyclic.h"
#include "prof.h"
#include "tables.h"

namespace mwj {
namespace {

struct CycPlan {
    uint32_t x, y, z;
    bool cbuckets() const { return x == 1 && y == 1; }   // R whole, C split (cyclic_c.cu)
};

struct CycLayout {
    uint2 *Rp, *Sp, *Tp;
    uint32_t *offR, *offS, *offT;
    uint32_t *items;
    void *scan_tmp;
    unsigned int *counter;
    unsigned long long *tile_rows, *tile_base;
    void *scan_tmp64;
    void *pscratch;
    size_t pscratch_bytes;
};

// shares (1, 1, z): R grouped by B, S and T by F(c)
struct CycCLayout {
    RGroup r;
    uint32_t *rmeta;
    unsigned int *hll, *bump;
    uint2 *Sp, *Tp;
    uint32_t *offS, *offT;
    uint32_t *items;
    void *scan_tmp;
    unsigned int *counter;
    unsigned long long *big_slots, *big_off, *bigset;
    uint32_t *bigcnt, *big_neg;
    unsigned long long *rep_set;   // the probe CTAs' regions for chunks that repeat (c, a) pairs
    uint32_t *rep_cnt;
    void *scan_tmp64b;
    unsigned long long *bucket_rows, *bucket_base;
    void *scan_tmp64;
    void *pscratch;
    size_t pscratch_bytes;
};

size_t cyc_c_layout(Arena &A, uint32_t z, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T, bool rows,
                    int num_sms, CycCLayout &L) {
    const size_t reserve = single_table_slots(R.n);
    L.rmeta = A.take<uint32_t>(kMetaWords);
    L.hll = A.take<unsigned int>(hll_scratch_registers(num_sms));
    L.bump = A.take<unsigned int>(1);
    L.r.meta = L.rmeta;
    L.r.keys = A.take<uint32_t>(reserve + 2);
    L.r.deg = A.take<uint32_t>(reserve + 2);
    L.r.end = A.take<uint32_t>(reserve + 2);
    L.r.alist = A.take<int32_t>(R.n + 4);
    L.Sp = A.take<uint2>(S.n + 2);
    L.offS = A.take<uint32_t>(z + 1);
    L.Tp = A.take<uint2>(T.n + 2);
    L.offT = A.take<uint32_t>(z + 1);
    L.items = A.take<uint32_t>(z + 1);
    L.scan_tmp = A.take<char>(scan_scratch_bytes(z + 1));
    L.counter = A.take<unsigned int>(1);
    L.big_slots = A.take<unsigned long long>(z + 1);
    L.big_off = A.take<unsigned long long>(z + 2);
    L.bigset = A.take<unsigned long long>(4 * (size_t)T.n + 16);
    L.bigcnt = A.take<uint32_t>(4 * (size_t)T.n + 16);
    L.rep_set = A.take<unsigned long long>(cyc_c_rep_slots(num_sms));
    L.rep_cnt = A.take<uint32_t>(cyc_c_rep_slots(num_sms));
    L.big_neg = A.take<uint32_t>(z + 1);
    L.scan_tmp64b = A.take<char>(scan_scratch_bytes(z + 1));
    if (rows) {
        L.bucket_rows = A.take<unsigned long long>(z + 1);
        L.bucket_base = A.take<unsigned long long>(z + 2);
        L.scan_tmp64 = A.take<char>(scan_scratch_bytes(z + 1));
    } else {
        L.bucket_rows = L.bucket_base = nullptr;
        L.scan_tmp64 = nullptr;
    }
    size_t ps = part_scratch_bytes(S.n, z, num_sms);
    const size_t ps2 = part_scratch_bytes(T.n, z, num_sms);
    if (ps2 > ps) ps = ps2;
    L.pscratch = A.take<char>(ps);
    L.pscratch_bytes = ps;
    return A.used;
}

size_t cyc_layout(Arena &A, const CycPlan &p, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                  bool rows, int num_sms, CycLayout &L) {
    const size_t ntiles = (size_t)p.x * p.y * p.z;
    L.Rp = A.take<uint2>(R.n + 2);
    L.offR = A.take<uint32_t>((size_t)p.x * p.y + 1);
    L.Sp = A.take<uint2>(S.n + 2);
    L.offS = A.take<uint32_t>((size_t)p.y * p.z + 1);
    L.Tp = A.take<uint2>(T.n + 2);
    L.offT = A.take<uint32_t>((size_t)p.z * p.x + 1);
    L.items = A.take<uint32_t>(ntiles + 1);
    L.scan_tmp = A.take<char>(scan_scratch_bytes(ntiles + 1));
    L.counter = A.take<unsigned int>(1);
    if (rows) {
        L.tile_rows = A.take<unsigned long long>(ntiles + 1);
        L.tile_base = A.take<unsigned long long>(ntiles + 2);
        L.scan_tmp64 = A.take<char>(scan_scratch_bytes(ntiles + 1));
    } else {
        L.tile_rows = L.tile_base = nullptr;
        L.scan_tmp64 = nullptr;
    }
    size_t ps = part_scratch_bytes(R.n, p.x * p.y, num_sms);
    size_t ps2 = part_scratch_bytes(S.n, p.y * p.z, num_sms);
    size_t ps3 = part_scratch_bytes(T.n, p.z * p.x, num_sms);
    if (ps2 > ps) ps = ps2;
    if (ps3 > ps) ps = ps3;
    L.pscratch = A.take<char>(ps);
    L.pscratch_bytes = ps;
    return A.used;
}

mwj_status check_cyc_shares(mwj_ctx *ctx, const mwj_shares &sh, CycPlan *p) {
    for (int k = 0; k < 3; ++k)
        if (sh.s[k] < 1) return fail(ctx, MWJ_ERR_INVALID_ARG, "shares must be >= 1");
    const uint64_t x = sh.s[0], y = sh.s[1], z = sh.s[2];
    if (x * y > kMaxBuckets || y * z > kMaxBuckets || z * x > kMaxBuckets)
        return fail(ctx, MWJ_ERR_INVALID_ARG, "cyclic shares: x*y, y*z, z*x must be <= %u",
                    kMaxBuckets);
    if (x * y * z > (1ull << 26))
        return fail(ctx, MWJ_ERR_INVALID_ARG, "cyclic shares: x*y*z must be <= 2^26");
    p->x = (uint32_t)x;
    p->y = (uint32_t)y;
    p->z = (uint32_t)z;
    return MWJ_OK;
}

}  // namespace

// Default shares: (1, 1, z), R whole and grouped by B, C split so that a
// bucket's T_k averages half of a CTA's on-chip set (cyclic_c.cu).  In the
// read cost z'|R| + x|S| + y|T| of Section 5.2 (with a third share) R is
// read once here, through the L2 as b -> [a] lists, and S and T once each;
// the cube tilings below keep R's buckets in shared memory instead.
mwj_status plan_cyclic_default(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                               mwj_shares *sh) {
    (void)ctx;
    (void)R;
    (void)S;
    const uint64_t want = ((uint64_t)T.n + cyc_c_tcap() / 2 - 1) / (cyc_c_tcap() / 2);
    uint32_t z = pow2_at_least(want ? want : 1);
    if (z > kMaxBuckets) z = kMaxBuckets;
    sh->s[0] = 1;
    sh->s[1] = 1;
    sh->s[2] = (int32_t)z;
    return MWJ_OK;
}

// Section 5.2 generalised to three shares: a tile (i,j,k) reads R_ij, S_jk
// and T_ki, so R is read z times, S x times and T y times; minimise
// z|R| + x|S| + y|T| over powers of two subject to the expected R_ij and
// T_ki fitting a CTA's tables with room to spare, and enough tiles to fill
// the GPU when the input is large.
mwj_status plan_cyclic_cube(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                            mwj_shares *sh) {
    const double nR = (double)R.n, nS = (double)S.n, nT = (double)T.n;
    const double rfit = 0.5 * cyc_rcap(), tfit = 0.5 * cyc_tcap();
    const bool big = nR + nS + nT > (double)(1 << 20);
    const double min_tiles = big ? 2.0 * ctx->dev.num_sms : 1.0;
    double best = INFINITY;
    uint32_t bx = 1, by = 1, bz = 1;
    for (uint32_t x = 1; x <= 4096; x <<= 1)
        for (uint32_t y = 1; y <= 4096; y <<= 1)
            for (uint32_t z = 1; z <= 4096; z <<= 1) {
                const uint64_t xy = (uint64_t)x * y, yz = (uint64_t)y * z, zx = (uint64_t)z * x;
                if (xy > kMaxBuckets || yz > kMaxBuckets || zx > kMaxBuckets) continue;
                if ((uint64_t)x * y * z > (1ull << 24)) continue;
                if (nR / xy > rfit || nT / zx > tfit) continue;
                if ((double)x * y * z < min_tiles) continue;
                const double cost = z * nR + x * nS + y * nT;
                if (cost < best) {
                    best = cost;
                    bx = x;
                    by = y;
                    bz = z;
                }
            }
    if (!std::isfinite(best)) {   // nothing fits the constraints: the largest legal tiling
        bx = 128;
        by = 256;
        bz = 128;
    }
    sh->s[0] = (int32_t)bx;
    sh->s[1] = (int32_t)by;
    sh->s[2] = (int32_t)bz;
    return MWJ_OK;
}

mwj_status cyc_workspace(mwj_ctx *ctx, const mwj_rel &R, const mwj_rel &S, const mwj_rel &T,
                         const mwj_shares *shares, mwj_mode mode, size_t *bytes) {
    mwj_shares sh;
    if (shares) sh = *shares; else plan_cyclic_default(ctx, R, S, T, &sh);
    CycPlan p;
    mwj_status s = check_cyc_shares(ctx, sh, &p);
    if (s != MWJ_OK) return s;
    Arena A(nullptr, 0);
    if (p.cbuckets()) {
        CycCLayout L;
        *bytes = cyc_c_layout(A, p.z, R, S, T, mode == MWJ_MATERIALIZE, ctx->dev.num_sms, L);
        return MWJ_OK;
    }
    CycLayout L;
    *bytes = cyc_layout(A, p, R, S, T, mode == MWJ_MATERIALIZE, ctx->dev.num_sms, L);
    return MWJ_OK;
}

}  // namespace mwj

using namespace mwj;

extern "C" mwj_status mwj_join3_cyclic(mwj_ctx *ctx, mwj_rel R, mwj_rel S, mwj_rel T,
                                       const mwj_shares *shares, const mwj_out *out,
                                       void *workspace, size_t ws_bytes, void *stream) {
    if (!ctx || !out) return MWJ_ERR_INVALID_ARG;
    ApiScope api_scope(&ctx->prof);
    if (!rel_ok(R) || !rel_ok(S) || !rel_ok(T)) return fail(ctx, MWJ_ERR_INVALID_ARG, "bad relation");
    mwj_status s = check_out(ctx, out, 3);
    if (s != MWJ_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    mwj_shares sh;
    if (shares) sh = *shares; else plan_cyclic_default(ctx, R, S, T, &sh);
    CycPlan p;
    if ((s = check_cyc_shares(ctx, sh, &p)) != MWJ_OK) return s;
    const bool rows = out->mode == MWJ_MATERIALIZE;
    Arena A(workspace, ws_bytes);
    CycLayout L;
    CycCLayout LC;
    if (p.cbuckets())
        cyc_c_layout(A, p.z, R, S, T, rows, ctx->dev.num_sms, LC);
    else
        cyc_layout(A, p, R, S, T, rows, ctx->dev.num_sms, L);
    if (A.overflow || !workspace)
        return fail(ctx, MWJ_ERR_WORKSPACE, "workspace of %zu bytes, %zu needed", ws_bytes, A.used);

    const Seeds &sd = ctx->seeds;
    cudaError_t e;
    if ((e = cudaMemsetAsync(out->total, 0, sizeof(int64_t), st)) != cudaSuccess)
        return cuda_fail(ctx, e, "memset total");
    if (out->mode == MWJ_COUNT_GROUP_BY_A &&
        (e = cudaMemsetAsync(out->group_counts, 0, sizeof(int64_t) * (size_t)out->a_domain, st)) !=
            cudaSuccess)
        return cuda_fail(ctx, e, "memset group_counts");
    if (p.cbuckets()) {
        // R grouped by B (every a checked against the group-by domain), then
        // S and T by F(c) into the same z buckets
        LC.r.seed = sd.slot;
        e = rgroup_build(R.x, R.y, R.n, LC.r, LC.hll, single_table_slots(R.n), LC.bump,
                         out->mode == MWJ_COUNT_GROUP_BY_A ? out->a_domain : 0, ctx->status, ctx->dev.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "group R by B");
        PartSpec ps{1, sd.C, p.z, -1, 0, 1};
        ps.st = ctx->status;
        e = part_run(S.x, S.y, S.n, ps, PAY_PAIR, LC.Sp, LC.offS, LC.pscratch, LC.pscratch_bytes,
                     ctx->dev.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "partition S");
        PartSpec pt{0, sd.C, p.z, -1, 0, 1};
        pt.st = ctx->status;
        e = part_run(T.x, T.y, T.n, pt, PAY_PAIR, LC.Tp, LC.offT, LC.pscratch, LC.pscratch_bytes,
                     ctx->dev.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "partition T");
        CycCArgs g{};
        g.r = LC.r;
        g.Sp = LC.Sp; g.offS = LC.offS; g.Tp = LC.Tp; g.offT = LC.offT;
        g.z = p.z;
        g.schunk = cyc_c_schunk(S.n, ctx->dev.num_sms);
        g.big_off = LC.big_off;
        g.bigset = LC.bigset;
        g.bigcnt = LC.bigcnt;
        g.big_neg = LC.big_neg;
        g.seed = sd.slot2;
        g.a_domain = out->a_domain;
        g.cnt = out->mode == MWJ_COUNT_GROUP_BY_A ? (unsigned long long *)out->group_counts : nullptr;
        g.total = (unsigned long long *)out->total;
        g.st = ctx->status;
        e = cyc_c_run(g, LC.items, LC.scan_tmp, LC.counter, LC.big_slots, LC.scan_tmp64b, LC.bucket_rows,
                      LC.bucket_base, LC.scan_tmp64, rows ? out->rows : nullptr, rows ? out->capacity : 0,
                      rows ? (long long *)out->n_rows : nullptr, LC.rep_set, LC.rep_cnt, ctx->dev.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cyclic probe");
        return MWJ_OK;
    }
    // Fig. 3: R by (H(a), G(b)), S by (G(b), F(c)), T by (F(c), H(a))
    PartSpec pr{0, sd.A, p.x, 1, sd.B, p.y};
    pr.st = ctx->status;
    if (out->mode == MWJ_COUNT_GROUP_BY_A) pr.dom = (uint32_t)out->a_domain;
    e = part_run(R.x, R.y, R.n, pr, PAY_PAIR, L.Rp, L.offR, L.pscratch, L.pscratch_bytes,
                 ctx->dev.num_sms, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "partition R");
    PartSpec ps{0, sd.B, p.y, 1, sd.C, p.z};
    ps.st = ctx->status;
    e = part_run(S.x, S.y, S.n, ps, PAY_PAIR, L.Sp, L.offS, L.pscratch, L.pscratch_bytes,
                 ctx->dev.num_sms, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "partition S");
    PartSpec pt{0, sd.C, p.z, 1, sd.A, p.x};
    pt.st = ctx->status;
    e = part_run(T.x, T.y, T.n, pt, PAY_PAIR, L.Tp, L.offT, L.pscratch, L.pscratch_bytes,
                 ctx->dev.num_sms, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "partition T");

    CycArgs g{};
    g.Rp = L.Rp; g.offR = L.offR; g.Sp = L.Sp; g.offS = L.offS; g.Tp = L.Tp; g.offT = L.offT;
    g.x = p.x; g.y = p.y; g.z = p.z;
    g.seed_slot = sd.slot;
    g.seed_slot2 = sd.slot2;
    g.a_domain = out->a_domain;
    g.cnt = out->mode == MWJ_COUNT_GROUP_BY_A ? (unsigned long long *)out->group_counts : nullptr;
    g.total = (unsigned long long *)out->total;
    g.st = ctx->status;
    e = cyc_run(g, L.items, L.scan_tmp, L.counter, L.tile_rows, L.tile_base, L.scan_tmp64,
                rows ? out->rows : nullptr, rows ? out->capacity : 0,
                rows ? (long long *)out->n_rows : nullptr, ctx->dev.num_sms, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cyclic probe");
    return MWJ_OK;
}
