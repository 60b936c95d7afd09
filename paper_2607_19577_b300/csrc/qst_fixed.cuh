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

struct FxSmem {
    int src, work, fbuf, stage, masks, meta, total;
};
// fbuf: dense c buffer (adjoint) or |.|^2 buffer (forward), floats at fx_pidx(u)
__host__ __device__ constexpr FxSmem fx_smem(bool adjoint) {
    FxSmem sp{};
    sp.src = 0;
    sp.work = sp.src + 8 * kFxBuf;
    sp.fbuf = sp.work + 8 * kFxBuf;
    sp.stage = sp.fbuf + 4 * kFxBuf;
    sp.masks = sp.stage + 2 * kStage * (adjoint ? 8 : 4);
    sp.meta = sp.masks + kMaxBin * (int)sizeof(uint2);
    sp.total = sp.meta + kMaxBin * (int)sizeof(SetMeta);
    return sp;
}
static_assert(fx_smem(true).masks % 16 == 0 && fx_smem(true).meta % 16 == 0, "aligned shared arrays");
static_assert(fx_smem(false).masks % 16 == 0 && fx_smem(false).meta % 16 == 0, "aligned shared arrays");
static_assert(2 * (fx_smem(true).total + 1024) <= 228 * 1024, "two units per SM");

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

// Forward unit = (bin, high pattern f, atom k), as k_forward, with fixed rounds.
__global__ void __launch_bounds__(kFxT, 2) k_forward_fx(const FwdArgs a) {
    constexpr FxSmem sp = fx_smem(false);
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *src = reinterpret_cast<float2 *>(smem + sp.src);
    float2 *work = reinterpret_cast<float2 *>(smem + sp.work);
    float *pbuf = reinterpret_cast<float *>(smem + sp.fbuf);
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem + sp.stage);
    uint2 *masks_sm = reinterpret_cast<uint2 *>(smem + sp.masks);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    const uint32_t tid = threadIdx.x;
    const int unit = blockIdx.x;
    const int k = unit % a.K;
    const int rest = unit / a.K;
    const uint32_t f = rest & ((1u << a.r) - 1u);
    const int bin = rest >> a.r;
    if (bin >= *a.n_bins) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    constexpr uint32_t cmask = 4095u;
    fx_stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, masks_sm, meta_sm);
    __syncthreads();
    const int bcount = b.count;
    const uint32_t *outcome = a.outcome;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            uint32_t *dst = stage + (si & 1) * kStage;
            const int nst = mt.cnt < kStage ? mt.cnt : kStage;
            for (int j = tid; j < nst; j += kFxT) cp_async4(dst + j, outcome + mt.lo + j);
        }
        cp_async_commit();
    };
    const float wk = a.w[k];
    float *pk = a.ppart + (size_t)k * a.nnz;
    issue(0);
    build_source<12, 4, true>(src, a.psi + (size_t)bin * a.src_bin_stride + (size_t)k * D, f, b.xytop, b.ytop, tid);
    __syncthreads();
    const uint32_t b0 = fx_pidx(fx_ubase<0>(tid)), b1 = fx_pidx(fx_ubase<1>(tid)), b2 = fx_pidx(fx_ubase<2>(tid));
    for (int si = 0; si < bcount; ++si) {
        issue(si + 1);
        const uint2 mk = masks_sm[si];
        const SetMeta mt = meta_sm[si];
        float2 v[16];
        fx_load<0>(v, src, b0);
        butterfly_fwd<4>(v, (mk.x >> 8) & 15u, (mk.y >> 8) & 15u);
        fx_store<0>(v, work, b0);  // every reader of work passed the previous setting's last barrier
        __syncthreads();
        fx_load<1>(v, work, b1);
        butterfly_fwd<4>(v, (mk.x >> 4) & 15u, (mk.y >> 4) & 15u);
        __syncwarp();
        fx_store<1>(v, work, b1);
        __syncwarp();
        fx_load<2>(v, work, b2);
        butterfly_fwd<4>(v, mk.x & 15u, mk.y & 15u);
        const float sc = wk * mt.cs;
#pragma unroll
        for (int i = 0; i < 16; ++i) pbuf[b2 + fx_roff<2>(i)] = sc * (v[i].x * v[i].x + v[i].y * v[i].y);
        cp_async_wait1();
        __syncthreads();
        const uint32_t *st = stage + (si & 1) * kStage;
        for (int j = tid; j < mt.cnt; j += kFxT) {
            const uint32_t u = (j < kStage ? st[j] : outcome[mt.lo + j]) & cmask;
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
}

// Adjoint unit = (bin, high pattern f, atom k), as k_adjoint, with fixed
// rounds: forward rounds 0, 1, 2, the c multiply in round 2's layout, inverse
// rounds 2, 1, 0 and the accumulator z in round 0's layout.
__global__ void __launch_bounds__(kFxT, 2) k_adjoint_fx(const AdjArgs a) {
    constexpr FxSmem sp = fx_smem(true);
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *src = reinterpret_cast<float2 *>(smem + sp.src);
    float2 *work = reinterpret_cast<float2 *>(smem + sp.work);
    float *cden = reinterpret_cast<float *>(smem + sp.fbuf);
    uint32_t *stage_u = reinterpret_cast<uint32_t *>(smem + sp.stage);
    float *stage_c = reinterpret_cast<float *>(smem + sp.stage + 2 * kStage * 4);
    uint2 *masks_sm = reinterpret_cast<uint2 *>(smem + sp.masks);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    const uint32_t tid = threadIdx.x;
    const int unit = blockIdx.x;
    const int k = unit % a.K;
    const int rest = unit / a.K;
    const uint32_t f = rest & ((1u << a.r) - 1u);
    const int bin = rest >> a.r;
    if (bin >= *a.n_bins) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    constexpr uint32_t cmask = 4095u;
    for (int u = tid; u < kFxBuf; u += kFxT) cden[u] = 0.f;
    fx_stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, masks_sm, meta_sm);
    __syncthreads();
    const int bcount = b.count;
    const uint32_t *outcome = a.outcome;
    const float *c_obs = a.c_obs;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            const int nst = mt.cnt < kStage ? mt.cnt : kStage;
            uint32_t *du = stage_u + (si & 1) * kStage;
            float *dc = stage_c + (si & 1) * kStage;
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
        const uint32_t *su = stage_u + (si & 1) * kStage;
        const float *sc = stage_c + (si & 1) * kStage;
        for (int j = tid; j < mt.cnt; j += kFxT) {
            const bool st = j < kStage;
            const uint32_t u = (st ? su[j] : outcome[mt.lo + j]) & cmask;
            cden[fx_pidx(u)] = clear ? 0.f : (st ? sc[j] : c_obs[mt.lo + j]) * mt.cs;
        }
    };
    issue(0);
    build_source<12, 4, true>(src, a.psi + (size_t)bin * a.src_bin_stride + (size_t)k * D, f, b.xytop, b.ytop, tid);
    cp_async_wait0();
    __syncthreads();  // c buffer zeroed, source built, first stage landed
    if (bcount > 0) scatter(0, false);
    const uint32_t b0 = fx_pidx(fx_ubase<0>(tid)), b1 = fx_pidx(fx_ubase<1>(tid)), b2 = fx_pidx(fx_ubase<2>(tid));
    float2 z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = make_float2(0.f, 0.f);
    for (int si = 0; si < bcount; ++si) {
        issue(si + 1);
        const uint2 mk = masks_sm[si];
        const uint32_t xy0 = (mk.x >> 8) & 15u, y0 = (mk.y >> 8) & 15u;
        const uint32_t xy1 = (mk.x >> 4) & 15u, y1 = (mk.y >> 4) & 15u;
        const uint32_t xy2 = mk.x & 15u, y2 = mk.y & 15u;
        float2 v[16];
        fx_load<0>(v, src, b0);
        butterfly_fwd<4>(v, xy0, y0);
        fx_store<0>(v, work, b0);
        __syncthreads();  // also publishes this setting's c scatter
        fx_load<1>(v, work, b1);
        butterfly_fwd<4>(v, xy1, y1);
        __syncwarp();
        fx_store<1>(v, work, b1);
        __syncwarp();
        fx_load<2>(v, work, b2);
        butterfly_fwd<4>(v, xy2, y2);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float cc = cden[b2 + fx_roff<2>(i)];
            v[i].x *= cc;
            v[i].y *= cc;
        }
        butterfly_inv<4>(v, xy2, y2);
        __syncwarp();
        fx_store<2>(v, work, b2);
        __syncwarp();
        fx_load<1>(v, work, b1);
        butterfly_inv<4>(v, xy1, y1);
        __syncwarp();
        fx_store<1>(v, work, b1);
        __syncthreads();  // every thread is also done reading the c buffer
        fx_load<0>(v, work, b0);
        butterfly_inv<4>(v, xy0, y0);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            z[i].x += v[i].x;
            z[i].y += v[i].y;
        }
        scatter(si, true);
        cp_async_wait0();
        __syncthreads();  // cleared before the next scatter; work and stage free for reuse
        if (si + 1 < bcount) scatter(si + 1, false);
    }
    float2 *zo = a.zbuf + ((size_t)bin * a.K + k) * D + ((size_t)f << 12);
#pragma unroll
    for (int i = 0; i < 16; ++i) zo[tid + (i << 8)] = z[i];
}
