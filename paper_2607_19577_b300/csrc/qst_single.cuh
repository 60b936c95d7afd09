// Single-setting chunk kernels for the wide path with 12-qubit chunks (n = 20;
// included inside qst.cu's anonymous namespace, after qst_fixed.cuh and
// qst_tensorcore.cuh).
//
// Every wide-path unit (setting j of a group, high pattern f, atom k) carries
// one setting, so there is nothing to amortise over settings: the source chunk
// goes straight into registers (round-0 layout of the three fixed rounds of
// qst_fixed.cuh), the rounds run, and z (adjoint) or the gather at the
// observed outcomes (forward) come from registers and the exchange buffer.
// A unit alone spends most of its time waiting: the source loads (32 KB from
// the group's intermediate, which is larger than L2), then the chain of
// metadata loads, then the outcome loads of the gather (ncu on the n = 20
// forward with one CTA per unit: 18.7 long-scoreboard stalls per issued
// instruction, DRAM at 24 % of peak; 1.21 ms per group against 0.57 ms here).
// So a CTA runs the units blockIdx.x, blockIdx.x + gridDim.x, ... and overlaps
// the next unit's loads with the current unit's rounds: one thread
// bulk-copies the next source chunk into shared memory (cp.async.bulk
// completing on an mbarrier) as soon as every thread has read the current one
// into registers, and the next unit's bin, setting, plan, CSR range and first
// outcomes are loaded in stages between the rounds.  The forward keeps the
// round-2 values in the exchange buffer and computes w 2^-m |.|^2 in the
// gather, so it needs no float buffer: 67 KB of shared memory, three CTAs per
// SM.  Every wait on the mbarrier is bounded: past the limit the CTA sets
// QST_DEV_TIMEOUT, waits (bounded) for the copy in flight and returns.

constexpr uint32_t kFx1pSrc = 4096u * 8u;  // one source chunk (complex64)
constexpr int kFx1pFwdSmem = kFxBuf * 8 + (int)kFx1pSrc + 16;
constexpr int kFx1pAdjSmem = kFxBuf * 12 + (int)kFx1pSrc + 16;
constexpr int kFx1pAdjcSmem = kFxBuf * 8;
static_assert(3 * (kFx1pFwdSmem + 1024) <= 228 * 1024 && 2 * (kFx1pAdjSmem + 1024) <= 228 * 1024,
              "three forward / two adjoint CTAs per SM");
static_assert((kFxBuf * 8) % 16 == 0 && (kFxBuf * 12) % 16 == 0, "the source buffer is 16-byte aligned");

__device__ __forceinline__ void fx1p_bulk(uint32_t dst, const void *src, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kFx1pSrc) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(kFx1pSrc), "r"(bar)
                 : "memory");
}

// A unit's setting: masks, 2^-m and its outcomes in chunk f (CSR range).
struct Fx1Unit {
    uint32_t xy, y;
    float cs;
    int64_t lo;
    int cnt;
};

// A unit of the wide path's grid: atom k, high pattern f, group-local bin.
struct Fx1Pos {
    int k, bin;
    uint32_t f;
};
__device__ __forceinline__ Fx1Pos fx1_pos(int unit, int K, int r) {
    Fx1Pos p;
    p.k = unit % K;
    const int rest = unit / K;
    p.f = rest & ((1u << r) - 1u);
    p.bin = rest >> r;
    return p;
}

// The next unit's metadata, loaded in three stages so that each dependent
// load has a round of work to arrive: the bin record, its setting, then the
// setting's plan and CSR range.
struct Fx1Next {
    Fx1Pos pos;
    Bin b;
    int s;
    Fx1Unit u;
};
__device__ __forceinline__ void fx1_stage1(Fx1Next &n, int unit, int K, int r, const Bin *__restrict__ bins) {
    n.pos = fx1_pos(unit, K, r);
    n.b = bins[n.pos.bin];
}
__device__ __forceinline__ void fx1_stage2(Fx1Next &n, const int32_t *__restrict__ order) { n.s = order[n.b.start]; }
__device__ __forceinline__ void fx1_stage3(Fx1Next &n, int nf, const SetPlan *__restrict__ plans,
                                           const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ choff) {
    const SetPlan &P = plans[n.s];
    n.u.xy = P.xy;
    n.u.y = P.y;
    n.u.cs = exp2f(-(float)P.m);
    const int32_t c0 = choff[(size_t)n.s * nf + n.pos.f], c1 = choff[(size_t)n.s * nf + n.pos.f + 1];
    n.u.lo = row_ptr[n.s] + c0;
    n.u.cnt = c1 - c0;
}

// Forward, persistent: per unit the three fixed rounds, then the gather at
// the observed outcomes (and, with CACHE, the store of the transforms).
template <bool CACHE>
__global__ void __launch_bounds__(kFxT, 3) k_forward_fx1p(const FwdArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *work = reinterpret_cast<float2 *>(smem);
    const float2 *sbuf = reinterpret_cast<const float2 *>(smem + kFxBuf * 8);
    const uint32_t s_src = smem_u32(smem + kFxBuf * 8), bar = s_src + kFx1pSrc;
    volatile int *abort_sm = reinterpret_cast<volatile int *>(smem + kFxBuf * 8 + kFx1pSrc + 8);
    const uint32_t tid = threadIdx.x;
    const int K = a.K, r = a.r, D = 1 << a.n, nf = (1 << r) + 1;
    const int total = (*a.n_bins << r) * K;
    int unit = blockIdx.x;
    if (unit >= total) return;
    constexpr uint32_t cmask = 4095u;
    auto src_of = [&](const Fx1Pos &p) {
        return a.psi + (size_t)p.bin * a.src_bin_stride + (size_t)p.k * D + ((size_t)p.f << 12);
    };
    Fx1Next cur;
    fx1_stage1(cur, unit, K, r, a.bins);
    if (tid == 0) {
        mb_init(bar);
        *abort_sm = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fx1p_bulk(s_src, src_of(cur.pos), bar);
    }
    fx1_stage2(cur, a.order);
    fx1_stage3(cur, nf, a.plans, a.row_ptr, a.choff);
    uint32_t out0 = (int)tid < cur.u.cnt ? a.outcome[cur.u.lo + tid] : 0u;
    __syncthreads();  // the barrier is initialised
    const uint32_t b0 = fx_pidx(fx_ubase<0>(tid)), b1 = fx_pidx(fx_ubase<1>(tid)), b2 = fx_pidx(fx_ubase<2>(tid));
    uint32_t phase = 0;
    for (;;) {
        const int next = unit + (int)gridDim.x;
        const bool has_next = next < total;
        if (!mb_wait(bar, phase)) *abort_sm = 1;
        float2 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sbuf[(i << 8) + tid];
        __syncthreads();  // every thread holds its source: the buffer may be refilled
        if (*abort_sm) break;
        phase ^= 1u;
        Fx1Next nx;
        if (has_next) {
            fx1_stage1(nx, next, K, r, a.bins);
            if (tid == 0) fx1p_bulk(s_src, src_of(nx.pos), bar);
        }
#pragma unroll
        for (int R = 0; R < 3; ++R) {
            butterfly_fwd<4>(v, fx_bits(cur.u.xy, R), fx_bits(cur.u.y, R));
            if (R < 2) fx_exchange(v, work, R, R + 1, b0, b1, b2);
            if (R == 0 && has_next) fx1_stage2(nx, a.order);
            if (R == 1 && has_next) fx1_stage3(nx, nf, a.plans, a.row_ptr, a.choff);
        }
        __syncwarp();  // the warp's round-2 reads of the exchange buffer are done
        fx_store<2>(v, work, b2);
        __syncthreads();  // the transforms are in the exchange buffer
        const float sc = a.w[cur.pos.k] * cur.u.cs;
        float *pk = a.ppart + (size_t)cur.pos.k * a.nnz;
        for (int j = tid; j < cur.u.cnt; j += kFxT) {
            const uint32_t u = (j == (int)tid ? out0 : a.outcome[cur.u.lo + j]) & cmask;
            const float2 ph = work[fx_pidx(u)];
            pk[cur.u.lo + j] = scaled_abs2(sc, ph);
            if (CACHE) a.phi_obs[(size_t)cur.pos.k * a.nnz + cur.u.lo + j] = ph;
        }
        if (a.p_dense) {
            float *pd = a.p_dense + (size_t)cur.s * D + ((size_t)cur.pos.f << 12);
            for (uint32_t u = tid; u <= cmask; u += kFxT) atomicAdd(pd + u, scaled_abs2(sc, work[fx_pidx(u)]));
        }
        if (!has_next) break;
        out0 = (int)tid < nx.u.cnt ? a.outcome[nx.u.lo + tid] : 0u;
        __syncthreads();  // the gather's reads of the exchange buffer are done
        unit = next;
        cur = nx;
    }
    if (*abort_sm && tid == 0) {  // the copy the failed wait was for may still land
        if (a.status) atomicOr(a.status, QST_DEV_TIMEOUT);
        mb_wait(bar, phase);
    }
}

// Adjoint that recomputes the rotations, persistent: per unit the dense c
// 2^-m, the forward rounds, the c multiply, the inverse rounds and z.
__global__ void __launch_bounds__(kFxT, 2) k_adjoint_fx1p(const AdjArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *work = reinterpret_cast<float2 *>(smem);
    float *cden = reinterpret_cast<float *>(smem + kFxBuf * 8);
    const float2 *sbuf = reinterpret_cast<const float2 *>(smem + kFxBuf * 12);
    const uint32_t s_src = smem_u32(smem + kFxBuf * 12), bar = s_src + kFx1pSrc;
    volatile int *abort_sm = reinterpret_cast<volatile int *>(smem + kFxBuf * 12 + kFx1pSrc + 8);
    const uint32_t tid = threadIdx.x;
    const int K = a.K, r = a.r, D = 1 << a.n, nf = (1 << r) + 1;
    const int total = (*a.n_bins << r) * K;
    int unit = blockIdx.x;
    if (unit >= total) return;
    constexpr uint32_t cmask = 4095u;
    auto src_of = [&](const Fx1Pos &p) {
        return a.psi + (size_t)p.bin * a.src_bin_stride + (size_t)p.k * D + ((size_t)p.f << 12);
    };
    Fx1Next cur;
    fx1_stage1(cur, unit, K, r, a.bins);
    if (tid == 0) {
        mb_init(bar);
        *abort_sm = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fx1p_bulk(s_src, src_of(cur.pos), bar);
    }
    fx1_stage2(cur, a.order);
    fx1_stage3(cur, nf, a.plans, a.row_ptr, a.choff);
    uint32_t out0 = 0u;
    float c0 = 0.f;
    if ((int)tid < cur.u.cnt) {
        out0 = a.outcome[cur.u.lo + tid];
        c0 = a.c_obs[cur.u.lo + tid];
    }
    for (int u = tid; u < kFxBuf; u += kFxT) cden[u] = 0.f;
    __syncthreads();  // the barrier is initialised, the c buffer zeroed
    const uint32_t b0 = fx_pidx(fx_ubase<0>(tid)), b1 = fx_pidx(fx_ubase<1>(tid)), b2 = fx_pidx(fx_ubase<2>(tid));
    uint32_t phase = 0;
    for (;;) {
        const int next = unit + (int)gridDim.x;
        const bool has_next = next < total;
        for (int j = tid; j < cur.u.cnt; j += kFxT) {
            const bool pre = j == (int)tid;
            cden[fx_pidx((pre ? out0 : a.outcome[cur.u.lo + j]) & cmask)] =
                (pre ? c0 : a.c_obs[cur.u.lo + j]) * cur.u.cs;
        }
        if (!mb_wait(bar, phase)) *abort_sm = 1;
        float2 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sbuf[(i << 8) + tid];
        __syncthreads();  // sources read, the scatter is visible
        if (*abort_sm) break;
        phase ^= 1u;
        Fx1Next nx;
        if (has_next) {
            fx1_stage1(nx, next, K, r, a.bins);
            if (tid == 0) fx1p_bulk(s_src, src_of(nx.pos), bar);
        }
#pragma unroll
        for (int R = 0; R < 3; ++R) {
            butterfly_fwd<4>(v, fx_bits(cur.u.xy, R), fx_bits(cur.u.y, R));
            if (R < 2) fx_exchange(v, work, R, R + 1, b0, b1, b2);
            if (R == 0 && has_next) fx1_stage2(nx, a.order);
            if (R == 1 && has_next) fx1_stage3(nx, nf, a.plans, a.row_ptr, a.choff);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float cc = cden[b2 + fx_roff<2>(i)];
            v[i].x = __fmul_rn(v[i].x, cc);  // not contracted into the butterflies that follow
            v[i].y = __fmul_rn(v[i].y, cc);
        }
#pragma unroll
        for (int R = 2; R >= 0; --R) {
            butterfly_inv<4>(v, fx_bits(cur.u.xy, R), fx_bits(cur.u.y, R));
            if (R > 0) fx_exchange(v, work, R, R - 1, b0, b1, b2);
        }
        float2 *zo = a.zbuf + ((size_t)cur.pos.bin * K + cur.pos.k) * D + ((size_t)cur.pos.f << 12);
#pragma unroll
        for (int i = 0; i < 16; ++i) zo[tid + (i << 8)] = v[i];
        if (!has_next) break;
        if ((int)tid < nx.u.cnt) {
            out0 = a.outcome[nx.u.lo + tid];
            c0 = a.c_obs[nx.u.lo + tid];
        }
        __syncthreads();  // every c value of this unit is read
        for (int j = tid; j < cur.u.cnt; j += kFxT) cden[fx_pidx(a.outcome[cur.u.lo + j] & cmask)] = 0.f;
        __syncthreads();  // cleared before the next scatter
        unit = next;
        cur = nx;
    }
    if (*abort_sm && tid == 0) {
        if (a.status) atomicOr(a.status, QST_DEV_TIMEOUT);
        mb_wait(bar, phase);
    }
}

// Adjoint from the stored transforms, persistent: per unit the scatter of
// y = c 2^-m phi into the zeroed exchange buffer, the inverse rounds and z.
// No source: only the metadata and the scattered values are prefetched.
__global__ void __launch_bounds__(kFxT, 4) k_adjoint_fx1cp(const AdjArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *work = reinterpret_cast<float2 *>(smem);
    const uint32_t tid = threadIdx.x;
    const int K = a.K, r = a.r, D = 1 << a.n, nf = (1 << r) + 1;
    const int total = (*a.n_bins << r) * K;
    int unit = blockIdx.x;
    if (unit >= total) return;
    constexpr uint32_t cmask = 4095u;
    Fx1Next cur;
    fx1_stage1(cur, unit, K, r, a.bins);
    fx1_stage2(cur, a.order);
    fx1_stage3(cur, nf, a.plans, a.row_ptr, a.choff);
    uint32_t out0 = 0u;
    float c0 = 0.f;
    float2 p0 = make_float2(0.f, 0.f);
    if ((int)tid < cur.u.cnt) {
        out0 = a.outcome[cur.u.lo + tid];
        c0 = a.c_obs[cur.u.lo + tid];
        p0 = a.phi_obs[(size_t)cur.pos.k * a.nnz + cur.u.lo + tid];
    }
    const uint32_t b0 = fx_pidx(fx_ubase<0>(tid)), b1 = fx_pidx(fx_ubase<1>(tid)), b2 = fx_pidx(fx_ubase<2>(tid));
    for (;;) {
        const int next = unit + (int)gridDim.x;
        const bool has_next = next < total;
        for (int u = tid; u < kFxBuf; u += kFxT) work[u] = make_float2(0.f, 0.f);
        __syncthreads();  // zeroed before any entry is scattered
        Fx1Next nx;
        if (has_next) fx1_stage1(nx, next, K, r, a.bins);
        const float2 *phk = a.phi_obs + (size_t)cur.pos.k * a.nnz;
        for (int j = tid; j < cur.u.cnt; j += kFxT) {
            const bool pre = j == (int)tid;
            const float cy = (pre ? c0 : a.c_obs[cur.u.lo + j]) * cur.u.cs;
            const float2 ph = pre ? p0 : phk[cur.u.lo + j];
            work[fx_pidx((pre ? out0 : a.outcome[cur.u.lo + j]) & cmask)] = make_float2(cy * ph.x, cy * ph.y);
        }
        __syncthreads();  // the scatter is visible
        if (has_next) fx1_stage2(nx, a.order);
        float2 v[16];
        fx_load<2>(v, work, b2);
#pragma unroll
        for (int R = 2; R >= 0; --R) {
            butterfly_inv<4>(v, fx_bits(cur.u.xy, R), fx_bits(cur.u.y, R));
            if (R > 0) fx_exchange(v, work, R, R - 1, b0, b1, b2);
            if (R == 2 && has_next) fx1_stage3(nx, nf, a.plans, a.row_ptr, a.choff);
            if (R == 1 && has_next && (int)tid < nx.u.cnt) {
                out0 = a.outcome[nx.u.lo + tid];
                c0 = a.c_obs[nx.u.lo + tid];
                p0 = a.phi_obs[(size_t)nx.pos.k * a.nnz + nx.u.lo + tid];
            }
        }
        float2 *zo = a.zbuf + ((size_t)cur.pos.bin * K + cur.pos.k) * D + ((size_t)cur.pos.f << 12);
#pragma unroll
        for (int i = 0; i < 16; ++i) zo[tid + (i << 8)] = v[i];
        if (!has_next) break;
        __syncthreads();  // the last exchange's loads are done before the zeroing
        unit = next;
        cur = nx;
    }
}
