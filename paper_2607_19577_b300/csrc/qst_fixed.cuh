// Fixed-position rounds for 12-qubit chunks (included inside qst.cu's
// anonymous namespace, after the generic chunk kernels).
//
// The generic kernels pick each round's register bits per setting (the X/Y
// positions), which needs a per-setting address walk: one XOR per amplitude
// per shared-memory pass.  Here the three rounds sit on fixed chunk-bit
// groups, so every address is a per-thread base plus a compile-time offset:
//
//   round 0: bits 8..11 in registers, thread bits 0..7
//   round 1: bits 4..7  in registers, thread bits 0..3, 8..11
//   round 2: bits 0..3  in registers, thread bits 4..11
//
// with 16 amplitudes per thread and 256 threads per unit.  Z bits inside a
// group are skipped by the butterflies as before (warp-uniform branches).
// Shared buffers use the padded index fx_pidx(u) = u + (u >> 4): it is
// additive over disjoint bit sets, and in every round the 16 lanes of a
// half-warp reach 16 distinct bank pairs (complex64) and a warp 32 distinct
// banks (float).  Rounds 1 and 2 both keep chunk bits 9..11 on the warp index,
// so the exchanges between them stay inside one warp (__syncwarp only): a
// setting costs three block barriers instead of about eight.

constexpr int kFxT = 256;                                    // threads per unit
constexpr int kFxBuf = (((int)fx_pidx(4095u) + 1 + 3) / 4) * 4;  // padded elements of a 2^12 chunk (x4)

// per-thread element index of register 0 in round R
template <int R>
__device__ __forceinline__ uint32_t fx_ubase(uint32_t t) {
    return R == 0 ? t : (R == 1 ? ((t & 15u) | ((t >> 4) << 8)) : (t << 4));
}
// padded offset of register element i in round R (compile-time)
template <int R>
__host__ __device__ constexpr uint32_t fx_roff(int i) {
    return fx_pidx(R == 0 ? (uint32_t)i << 8 : (R == 1 ? (uint32_t)i << 4 : (uint32_t)i));
}

template <int R>
__device__ __forceinline__ void fx_load(float2 (&v)[16], const float2 *buf, uint32_t base) {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = buf[base + fx_roff<R>(i)];
}
template <int R>
__device__ __forceinline__ void fx_store(const float2 (&v)[16], float2 *buf, uint32_t base) {
#pragma unroll
    for (int i = 0; i < 16; ++i) buf[base + fx_roff<R>(i)] = v[i];
}

// Tensor memory holds what a unit keeps across its settings: the source chunk
// (round-0 layout, 32 columns per thread) and, in the adjoint, the
// accumulator z (32 more).  Warp w owns TMEM lanes 32 (w mod 4) + lane and
// column block w / 4, so each thread reads and writes only its own lane.  That
// takes the source off the shared-memory pipe (one tcgen05.ld per setting
// instead of 16 LDS) and frees the shared memory and registers that allow
// three units per SM.
constexpr int kFxStage = 512;   // observed entries per setting staged by cp.async
constexpr uint32_t kFxColsFwd = 64, kFxColsAdj = 128;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// warp-wide: allocate ncols TMEM columns, base address written to *dst
__device__ __forceinline__ void tm_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

#define QST_R32(v) \
    v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8], v[9], v[10], v[11], v[12], v[13], v[14], v[15], v[16], \
        v[17], v[18], v[19], v[20], v[21], v[22], v[23], v[24], v[25], v[26], v[27], v[28], v[29], v[30], v[31]
#define QST_OPS32(c)                                                                                              \
    c(r[0]), c(r[1]), c(r[2]), c(r[3]), c(r[4]), c(r[5]), c(r[6]), c(r[7]), c(r[8]), c(r[9]), c(r[10]), c(r[11]), \
        c(r[12]), c(r[13]), c(r[14]), c(r[15]), c(r[16]), c(r[17]), c(r[18]), c(r[19]), c(r[20]), c(r[21]),      \
        c(r[22]), c(r[23]), c(r[24]), c(r[25]), c(r[26]), c(r[27]), c(r[28]), c(r[29]), c(r[30]), c(r[31])
#define QST_OUT(x) "=r"(x)
#define QST_INOUT(x) "+r"(x)
#define QST_IN(x) "r"(x)

// 32 consecutive columns of this thread's lane <-> 16 complex values (re, im).
// tm_ld_issue starts the load; tm_ld_wait completes it and ties the registers
// to the completion, so no use can be scheduled before it.
__device__ __forceinline__ void tm_ld_issue(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : QST_OPS32(QST_OUT)
        : "r"(taddr));
}
__device__ __forceinline__ void tm_ld_wait(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : QST_OPS32(QST_INOUT)::"memory");
}
__device__ __forceinline__ void tm_st(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        QST_OPS32(QST_IN)
        : "memory");
}
#define QST_OPS16(c)                                                                                              \
    c(r[0]), c(r[1]), c(r[2]), c(r[3]), c(r[4]), c(r[5]), c(r[6]), c(r[7]), c(r[8]), c(r[9]), c(r[10]), c(r[11]), \
        c(r[12]), c(r[13]), c(r[14]), c(r[15])
// the same for 16 columns (8 complex values)
__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : QST_OPS16(QST_OUT)
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : QST_OPS16(QST_INOUT)::"memory");
}
__device__ __forceinline__ void tm_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        QST_OPS16(QST_IN)
        : "memory");
}

__device__ __forceinline__ void to_words(const float2 (&v)[16], uint32_t (&r)[32]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        r[2 * i] = __float_as_uint(v[i].x);
        r[2 * i + 1] = __float_as_uint(v[i].y);
    }
}
__device__ __forceinline__ void from_words(const uint32_t (&r)[32], float2 (&v)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
}

struct FxSmem {
    int work, fbuf, stage, masks, meta, tmem, total;
};
// fbuf: dense c buffer (adjoint) or |.|^2 buffer (forward), floats at fx_pidx(u)
__host__ __device__ constexpr FxSmem fx_smem(bool adjoint) {
    FxSmem sp{};
    sp.work = 0;
    sp.fbuf = sp.work + 8 * kFxBuf;
    sp.stage = sp.fbuf + 4 * kFxBuf;
    sp.masks = sp.stage + 2 * kFxStage * (adjoint ? 8 : 4);
    sp.meta = sp.masks + kMaxBin * (int)sizeof(uint2);
    sp.tmem = sp.meta + kMaxBin * (int)sizeof(SetMeta);
    sp.total = sp.tmem + 16;
    return sp;
}
static_assert(fx_smem(true).masks % 16 == 0 && fx_smem(true).meta % 16 == 0, "aligned shared arrays");
static_assert(fx_smem(false).masks % 16 == 0 && fx_smem(false).meta % 16 == 0, "aligned shared arrays");
static_assert(3 * (fx_smem(true).total + 1024) <= 228 * 1024, "three units per SM");
// at most four units of either kind fit on an SM (shared memory), and their
// TMEM columns then fit in the SM's 512: no allocation ever waits
static_assert(5 * (fx_smem(false).total + 1024) > 228 * 1024 && 4 * kFxColsAdj <= 512, "TMEM never oversubscribed");

// Stage a bin's (xy, y) masks and chunk-f ranges in shared memory (the fixed
// rounds need nothing else from the setting plans).
__device__ __forceinline__ void fx_stage_bin(const Bin &b, uint32_t f, int nf, const int32_t *__restrict__ order,
                                             const SetPlan *__restrict__ plans, const int64_t *__restrict__ row_ptr,
                                             const int32_t *__restrict__ choff, uint2 *masks_sm, SetMeta *meta_sm) {
    for (int si = threadIdx.x; si < b.count; si += blockDim.x) {
        const int s = order[b.start + si];
        const SetPlan &P = plans[s];
        masks_sm[si] = make_uint2(P.xy, P.y);
        const int64_t rb = row_ptr[s];
        const int32_t c0 = choff[(size_t)s * nf + f], c1 = choff[(size_t)s * nf + f + 1];
        SetMeta mt;
        mt.lo = (int32_t)(rb + c0);
        mt.cnt = c1 - c0;
        mt.off = 0;
        mt.cs = exp2f(-(float)P.m);
        meta_sm[si] = mt;
    }
}

// Round R's butterflies (forward or inverse) act on the chunk bits
// 4 (2 - R) .. 4 (2 - R) + 3 of the setting's masks.  The round loops are
// unrolled: the exchanges then resolve at compile time (measured faster than
// one butterfly site per direction, despite the larger code).
__device__ __forceinline__ uint32_t fx_bits(uint32_t mask, int R) { return (mask >> (8 - 4 * R)) & 15u; }

// Exchanges between rounds.  Round 0 <-> 1 crosses warps (block barrier after
// the stores); round 1 <-> 2 stays inside a warp.  Every exchange starts with
// a warp barrier: the warp's previous reads of the same addresses are done,
// and for the cross-warp stores the block barrier at the end of the previous
// exchange or setting already separates other warps' reads.
__device__ __forceinline__ void fx_exchange(float2 (&v)[16], float2 *work, int from, int to, uint32_t b0, uint32_t b1,
                                            uint32_t b2) {
    __syncwarp();
    if (from == 0) fx_store<0>(v, work, b0);
    else if (from == 1) fx_store<1>(v, work, b1);
    else fx_store<2>(v, work, b2);
    if (from == 0 || to == 0) __syncthreads();
    else __syncwarp();
    if (to == 0) fx_load<0>(v, work, b0);
    else if (to == 1) fx_load<1>(v, work, b1);
    else fx_load<2>(v, work, b2);
}

// Forward unit = (bin, high pattern f, atom k), as k_forward, with fixed rounds.
__device__ __forceinline__ void forward_fx_body(const FwdArgs a, const int cta) {
    constexpr FxSmem sp = fx_smem(false);
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *work = reinterpret_cast<float2 *>(smem + sp.work);
    float *pbuf = reinterpret_cast<float *>(smem + sp.fbuf);
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem + sp.stage);
    uint2 *masks_sm = reinterpret_cast<uint2 *>(smem + sp.masks);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    uint32_t *tmem_sm = reinterpret_cast<uint32_t *>(smem + sp.tmem);
    const uint32_t tid = threadIdx.x, warp = tid >> 5;
    const int unit = cta;
    const int k = unit % a.K;
    const int rest = unit / a.K;
    const uint32_t f = rest & ((1u << a.r) - 1u);
    const int bin = rest >> a.r;
    if (bin >= *a.n_bins || (a.skip && *a.skip)) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    constexpr uint32_t cmask = 4095u;
    if (warp == 0) tm_alloc(tmem_sm, kFxColsFwd);
    fx_stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, masks_sm, meta_sm);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t t_src = tmem_sm[0] + (((warp & 3u) * 32u) << 16) + (warp >> 2) * 32u;
    const int bcount = b.count;
    const uint32_t *outcome = a.outcome;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            uint32_t *dst = stage + (si & 1) * kFxStage;
            const int nst = mt.cnt < kFxStage ? mt.cnt : kFxStage;
            for (int j = tid; j < nst; j += kFxT) cp_async4(dst + j, outcome + mt.lo + j);
        }
        cp_async_commit();
    };
    const float wk = a.w[k];
    float *pk = a.ppart + (size_t)k * a.nnz;
    issue(0);
    {
        float2 acc[16];
        const float2 *psik = a.psi + (size_t)bin * a.src_bin_stride + (size_t)k * D;
        build_source_regs<12, 4, 0, 8>(acc, psik, f, b.xytop, b.ytop, tid);
        build_source_regs<12, 4, 8, 8>(acc, psik, f, b.xytop, b.ytop, tid);
        uint32_t r[32];
        to_words(acc, r);
        tm_st(t_src, r);
        tm_wait_st();
    }
    const uint32_t b0 = fx_pidx(fx_ubase<0>(tid)), b1 = fx_pidx(fx_ubase<1>(tid)), b2 = fx_pidx(fx_ubase<2>(tid));
    for (int si = 0; si < bcount; ++si) {
        issue(si + 1);
        const uint2 mk = masks_sm[si];
        const SetMeta mt = meta_sm[si];
        float2 v[16];
        {
            uint32_t r[32];
            tm_ld_issue(t_src, r);
            tm_ld_wait(r);
            from_words(r, v);
        }
#pragma unroll
        for (int R = 0; R < 3; ++R) {
            butterfly_fwd<4>(v, fx_bits(mk.x, R), fx_bits(mk.y, R));
            if (R < 2) fx_exchange(v, work, R, R + 1, b0, b1, b2);
        }
        const float sc = wk * mt.cs;
#pragma unroll
        for (int i = 0; i < 16; ++i) pbuf[b2 + fx_roff<2>(i)] = scaled_abs2(sc, v[i]);
        cp_async_wait1();
        __syncthreads();
        const uint32_t *st = stage + (si & 1) * kFxStage;
        for (int j = tid; j < mt.cnt; j += kFxT) {
            const uint32_t u = (j < kFxStage ? st[j] : outcome[mt.lo + j]) & cmask;
            pk[mt.lo + j] = pbuf[fx_pidx(u)];
        }
        if (a.p_dense) {
            const int s = a.order[b.start + si];
            float *pd = a.p_dense + (size_t)s * D + ((size_t)f << 12);
            for (uint32_t u = tid; u <= cmask; u += kFxT) atomicAdd(pd + u, pbuf[fx_pidx(u)]);
        }
        __syncthreads();  // pbuf, work and the stage buffer are reused by the next setting
    }
    cp_async_wait0();
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(tmem_sm[0], kFxColsFwd);
    }
}
__global__ void __launch_bounds__(kFxT, 3) k_forward_fx(const FwdArgs a) {
    forward_fx_body(a, blockIdx.x);
}
__global__ void __launch_bounds__(kFxT, 3) k_forward_fx_multi(const FwdArgs *__restrict__ args, const int *__restrict__ start, int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const FwdArgs a = args[i];
    forward_fx_body(a, (int)blockIdx.x - start[i]);
}

// Adjoint unit = (bin, high pattern f, atom k), as k_adjoint, with fixed
// rounds: forward rounds 0, 1, 2, the c multiply in round 2's layout, inverse
// rounds 2, 1, 0 and the accumulator z (TMEM) in round 0's layout.
__device__ __forceinline__ void adjoint_fx_body(const AdjArgs a, const int cta) {
    if (a.skip && *a.skip) return;
    constexpr FxSmem sp = fx_smem(true);
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *work = reinterpret_cast<float2 *>(smem + sp.work);
    float *cden = reinterpret_cast<float *>(smem + sp.fbuf);
    uint32_t *stage_u = reinterpret_cast<uint32_t *>(smem + sp.stage);
    float *stage_c = reinterpret_cast<float *>(smem + sp.stage + 2 * kFxStage * 4);
    uint2 *masks_sm = reinterpret_cast<uint2 *>(smem + sp.masks);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    uint32_t *tmem_sm = reinterpret_cast<uint32_t *>(smem + sp.tmem);
    const uint32_t tid = threadIdx.x, warp = tid >> 5;
    const int unit = cta;
    const int k = unit % a.K;
    const int rest = unit / a.K;
    const uint32_t f = rest & ((1u << a.r) - 1u);
    const int bin = rest >> a.r;
    if (bin >= *a.n_bins) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    constexpr uint32_t cmask = 4095u;
    if (warp == 0) tm_alloc(tmem_sm, kFxColsAdj);
    for (int u = tid; u < kFxBuf; u += kFxT) cden[u] = 0.f;
    fx_stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, masks_sm, meta_sm);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t t_src = tmem_sm[0] + (((warp & 3u) * 32u) << 16) + (warp >> 2) * 32u;
    const uint32_t t_z = t_src + 64u;
    const int bcount = b.count;
    const uint32_t *outcome = a.outcome;
    const float *c_obs = a.c_obs;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            const int nst = mt.cnt < kFxStage ? mt.cnt : kFxStage;
            uint32_t *du = stage_u + (si & 1) * kFxStage;
            float *dc = stage_c + (si & 1) * kFxStage;
            for (int j = tid; j < nst; j += kFxT) {
                cp_async4(du + j, outcome + mt.lo + j);
                cp_async4(dc + j, c_obs + mt.lo + j);
            }
        }
        cp_async_commit();
    };
    // scatter (c 2^-m) or clear setting si's entries of the dense c buffer;
    // each thread touches the entries it staged itself
    auto scatter = [=](int si, bool clear) {
        const SetMeta mt = meta_sm[si];
        const uint32_t *su = stage_u + (si & 1) * kFxStage;
        const float *sc = stage_c + (si & 1) * kFxStage;
        for (int j = tid; j < mt.cnt; j += kFxT) {
            const bool st = j < kFxStage;
            const uint32_t u = (st ? su[j] : outcome[mt.lo + j]) & cmask;
            cden[fx_pidx(u)] = clear ? 0.f : (st ? sc[j] : c_obs[mt.lo + j]) * mt.cs;
        }
    };
    issue(0);
    {
        float2 acc[16];
        const float2 *psik = a.psi + (size_t)bin * a.src_bin_stride + (size_t)k * D;
        build_source_regs<12, 4, 0, 8>(acc, psik, f, b.xytop, b.ytop, tid);
        build_source_regs<12, 4, 8, 8>(acc, psik, f, b.xytop, b.ytop, tid);
        uint32_t r[32];
        to_words(acc, r);
        tm_st(t_src, r);
#pragma unroll
        for (int i = 0; i < 32; ++i) r[i] = 0u;
        tm_st(t_z, r);
        tm_wait_st();
    }
    cp_async_wait0();
    __syncthreads();  // c buffer zeroed, first stage landed
    if (bcount > 0) scatter(0, false);
    const uint32_t b0 = fx_pidx(fx_ubase<0>(tid)), b1 = fx_pidx(fx_ubase<1>(tid)), b2 = fx_pidx(fx_ubase<2>(tid));
    for (int si = 0; si < bcount; ++si) {
        issue(si + 1);
        const uint2 mk = masks_sm[si];
        float2 v[16];
        {
            uint32_t r[32];
            tm_ld_issue(t_src, r);
            tm_ld_wait(r);
            from_words(r, v);
        }
        // forward rounds 0, 1, 2 (the first block barrier also publishes this setting's c scatter)
#pragma unroll
        for (int R = 0; R < 3; ++R) {
            butterfly_fwd<4>(v, fx_bits(mk.x, R), fx_bits(mk.y, R));
            if (R < 2) fx_exchange(v, work, R, R + 1, b0, b1, b2);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float cc = cden[b2 + fx_roff<2>(i)];
            v[i].x = __fmul_rn(v[i].x, cc);  // not contracted into the butterflies that follow
            v[i].y = __fmul_rn(v[i].y, cc);
        }
        // inverse rounds 2, 1, 0 (the block barrier of 1 -> 0 also ends every read of the c buffer)
#pragma unroll
        for (int R = 2; R >= 0; --R) {
            butterfly_inv<4>(v, fx_bits(mk.x, R), fx_bits(mk.y, R));
            if (R > 0) fx_exchange(v, work, R, R - 1, b0, b1, b2);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // z += v, eight complex values at a time
            uint32_t r[16];
            tm_ld16(t_z + 16u * h, r);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                r[2 * i] = __float_as_uint(__uint_as_float(r[2 * i]) + v[8 * h + i].x);
                r[2 * i + 1] = __float_as_uint(__uint_as_float(r[2 * i + 1]) + v[8 * h + i].y);
            }
            tm_st16(t_z + 16u * h, r);
        }
        tm_wait_st();
        scatter(si, true);
        cp_async_wait0();
        __syncthreads();  // cleared before the next scatter; work and stage free for reuse
        if (si + 1 < bcount) scatter(si + 1, false);
    }
    {
        uint32_t r[32];
        tm_ld_issue(t_z, r);
        tm_ld_wait(r);
        float2 *zo = a.zbuf + ((size_t)bin * a.K + k) * D + ((size_t)f << 12);
#pragma unroll
        for (int i = 0; i < 16; ++i) zo[tid + (i << 8)] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
    }
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(tmem_sm[0], kFxColsAdj);
    }
}
__global__ void __launch_bounds__(kFxT, 3) k_adjoint_fx(const AdjArgs a) {
    adjoint_fx_body(a, blockIdx.x);
}
__global__ void __launch_bounds__(kFxT, 3) k_adjoint_fx_multi(const AdjArgs *__restrict__ args, const int *__restrict__ start, int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const AdjArgs a = args[i];
    adjoint_fx_body(a, (int)blockIdx.x - start[i]);
}
