// Two-round kernels for 12-qubit chunks (included inside qst.cu's anonymous
// namespace, after qst_fixed.cuh).
//
// A 2^12 chunk is a 64 x 64 array u = lo + 64 hi, and each round transforms
// six of its qubits with 64 amplitudes per thread:
//
//   round A: chunk bits 6..11 in registers (element i = hi), thread t = lo
//   round B: chunk bits 0..5  in registers (element j = lo), thread t = hi
//
// so the forward pass needs one shared-memory exchange per setting (A -> B)
// and the adjoint two (A -> B after the forward round A, B -> A before the
// inverse round A), half of what three 4-bit rounds need.  A CTA runs two
// atoms, k0 = 2 kp (warps 0-1) and k0 + 1 (warps 2-3), on the same bin and
// high pattern: they share the staged setting metadata (and, in the adjoint,
// the dense c buffer), and the four warps reach all 128 TMEM lanes.  This file
// holds the forward kernel on scalar complex registers; the adjoint kernel,
// on packed FP32 pairs, is in qst_tworound_packed.cuh.
//
// Chunks of C = 10 or 11 qubits (whole states of 10, 11 qubits) keep 64
// amplitudes per thread with 2^(C-6) threads per atom (TA = C - 6 thread
// bits), so a CTA of 128 threads runs 2^(13-C) atoms:
//
//   round A: chunk bits TA..TA+5 in registers (element i), thread t = bits
//            0..TA-1 (amplitude t + 2^TA i); it transforms bits 6..C-1 only
//   round B: chunk bits 0..5 in registers, thread t = bits 6..C-1
//
// (chunk bits TA..5 sit in both rounds' registers; round B transforms them).
// The exchange buffer keeps u at row u / 64, column u mod 64.
//
// Exchange buffer (one per atom): u at 66 hi + lo.  Round-A accesses (lanes
// over lo) are contiguous; round-B accesses (lanes over hi, pairs of lo as
// one 16-byte access) are aligned, and the 8 lanes of each quarter-warp reach
// distinct 16-byte bank groups (66 hi / 2 = 33 hi, odd).
// Float buffers (dense c, w |.|^2): u at 68 hi + lo, read and written as
// float4 in round B's layout (17 hi + quad: distinct bank groups).  Both
// paddings are additive over (hi, lo), so every register element is a
// compile-time offset from one per-thread base.

constexpr int k2T = 128;                 // threads per CTA (two atoms of 64)
constexpr int k2Row = 66;                // complex elements per padded row of the exchange buffer
constexpr int k2Buf = 64 * k2Row;        // complex elements of one atom's exchange buffer
constexpr int k2FRow = 68;               // floats per padded row of a float buffer
constexpr int k2FBuf = 64 * k2FRow;      // floats of one float buffer
constexpr int k2Stage = 512;             // observed entries per setting staged by cp.async
constexpr uint32_t k2ColsFwd = 128;     // TMEM columns of a forward CTA: the source

__host__ __device__ constexpr uint32_t k2_fpos(uint32_t u) { return u + 4u * (u >> 6); }

struct K2Smem {
    int work, fbuf, stage, masks, meta, tmem, total;
};
// The forward writes w |.|^2 into each atom's exchange buffer once the
// exchange is read, so it has no float buffer of its own (fbuf = stage).
__host__ __device__ constexpr K2Smem k2_smem_fwd() {
    K2Smem sp{};
    sp.work = 0;
    sp.fbuf = sp.work + 2 * k2Buf * 8;
    sp.stage = sp.fbuf;
    sp.masks = sp.stage + 2 * k2Stage * 4;
    sp.meta = sp.masks + kMaxBin * (int)sizeof(uint2);
    sp.tmem = sp.meta + kMaxBin * (int)sizeof(SetMeta);
    sp.total = sp.tmem + 16;
    return sp;
}
static_assert(k2_smem_fwd().fbuf % 16 == 0 && k2_smem_fwd().masks % 16 == 0 && k2_smem_fwd().meta % 16 == 0,
              "aligned shared arrays");
static_assert(k2FBuf * 4 <= k2Buf * 8, "a float buffer fits in an exchange buffer");
constexpr int k2SmemSM = 228 * 1024;  // shared memory per SM; each CTA also reserves 1 KB
constexpr int k2CtaFwd = k2_smem_fwd().total + 1024;
static_assert(3 * k2CtaFwd <= k2SmemSM && 4 * k2CtaFwd > k2SmemSM, "three forward CTAs per SM");

// named barrier of the 64 threads of one atom (ids 1, 2; 0 is __syncthreads).
// Immediate ids (half is warp-uniform) keep the CTA's barrier count at three.
__device__ __forceinline__ void k2_bar_atom(uint32_t half) {
    if (half) asm volatile("bar.sync 2, 64;" ::: "memory");
    else asm volatile("bar.sync 1, 64;" ::: "memory");
}

// 128 consecutive TMEM columns of this thread's lane -> 64 complex values,
// loaded straight into v's registers: k2_tm_ld64_issue starts the four loads,
// k2_tm_ld64_wait completes them and ties every register of v to the
// completion, so no use is scheduled before it.  Work placed between the two
// hides the load latency.
#define QST_V16(c, o)                                                                                          \
    c(v[o + 0].x), c(v[o + 0].y), c(v[o + 1].x), c(v[o + 1].y), c(v[o + 2].x), c(v[o + 2].y), c(v[o + 3].x),    \
        c(v[o + 3].y), c(v[o + 4].x), c(v[o + 4].y), c(v[o + 5].x), c(v[o + 5].y), c(v[o + 6].x), c(v[o + 6].y), \
        c(v[o + 7].x), c(v[o + 7].y), c(v[o + 8].x), c(v[o + 8].y), c(v[o + 9].x), c(v[o + 9].y), c(v[o + 10].x), \
        c(v[o + 10].y), c(v[o + 11].x), c(v[o + 11].y), c(v[o + 12].x), c(v[o + 12].y), c(v[o + 13].x),         \
        c(v[o + 13].y), c(v[o + 14].x), c(v[o + 14].y), c(v[o + 15].x), c(v[o + 15].y)
#define QST_FOUT(x) "=f"(x)
#define QST_FINOUT(x) "+f"(x)
template <int Q>
__device__ __forceinline__ void k2_tm_ld16_issue(uint32_t taddr, float2 (&v)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : QST_V16(QST_FOUT, 16 * Q)
        : "r"(taddr + 32u * Q));
}
template <int Q>
__device__ __forceinline__ void k2_tm_ld16_tie(float2 (&v)[64]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : QST_V16(QST_FINOUT, 16 * Q)::"memory");
}
__device__ __forceinline__ void k2_tm_ld64_issue(uint32_t taddr, float2 (&v)[64]) {
    k2_tm_ld16_issue<0>(taddr, v);
    k2_tm_ld16_issue<1>(taddr, v);
    k2_tm_ld16_issue<2>(taddr, v);
    k2_tm_ld16_issue<3>(taddr, v);
}
__device__ __forceinline__ void k2_tm_ld64_wait(float2 (&v)[64]) {
    k2_tm_ld16_tie<0>(v);
    k2_tm_ld16_tie<1>(v);
    k2_tm_ld16_tie<2>(v);
    k2_tm_ld16_tie<3>(v);
}
__device__ __forceinline__ void k2_tm_ld64(uint32_t taddr, float2 (&v)[64]) {
    k2_tm_ld64_issue(taddr, v);
    k2_tm_ld64_wait(v);
}
// elements 16 q .. 16 q + 15 of v -> TMEM columns 32 q .. 32 q + 31
template <int Q>
__device__ __forceinline__ void k2_tm_st16(uint32_t taddr, const float2 (&v)[64]) {
    uint32_t r[32];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        r[2 * i] = __float_as_uint(v[16 * Q + i].x);
        r[2 * i + 1] = __float_as_uint(v[16 * Q + i].y);
    }
    tm_st(taddr + 32u * Q, r);
}
// Chunk f of (U_h (x) I) psi_k in round A's layout (element i of thread t =
// amplitude t + 2^(C-6) i) -> TMEM columns 0..127, built 16 elements at a time.
// An inactive atom (k >= K) gets zeros.  CS > C: one 2^C block of a chunk of
// CS bits (psik points at the block's offset inside chunk 0).
template <int C = 12, int CS = C>
__device__ __forceinline__ void k2_build_source(uint32_t t_src, const float2 *psik, bool active, uint32_t f,
                                                uint32_t xytop, uint32_t ytop, uint32_t t) {
    float2 acc[64];
#define QST_K2_PART(Q)                                                                   \
    if (active) {                                                                        \
        build_source_regs<C, 6, 16 * (Q), 16, CS>(acc, psik, f, xytop, ytop, t);         \
    } else {                                                                             \
        _Pragma("unroll") for (int i = 0; i < 16; ++i) acc[16 * (Q) + i] = make_float2(0.f, 0.f); \
    }                                                                                    \
    k2_tm_st16<Q>(t_src, acc);
    QST_K2_PART(0)
    QST_K2_PART(1)
    QST_K2_PART(2)
    QST_K2_PART(3)
#undef QST_K2_PART
}

// Chunk factors of the two-round kernels, unscaled and in place:
//   X:  (a, b) -> (a + b, a - b)             as  a += b;  b = a - 2b
//   Y:  (a, b) -> (a - i b, i a - b)         as  a -= i b; b = i a - 2b
// The Y rows are those of V_Y = [[1,-i],[1,i]]/sqrt2 with the second row
// multiplied by i.  A per-outcome phase changes neither |(V_s psi)_u|^2 nor
// V_s^* (c .* V_s psi) (diagonals commute), and with it both factors are
// Hermitian and square to 2 I: the conjugate-transposed chunk transform is
// the chunk transform itself, so the adjoint's inverse rounds run the same
// butterfly code as its forward rounds.  (The high-bit factors, applied when
// the source chunk is built and by k_reduce, keep their own convention; they
// are separate tensor factors.)
template <int A>
__device__ __forceinline__ void butterfly_herm(float2 (&v)[1 << A], uint32_t xyf, uint32_t yf) {
#pragma unroll
    for (int j = 0; j < A; ++j) {
        if (!((xyf >> j) & 1u)) continue;
        if ((yf >> j) & 1u) {
#pragma unroll
            for (int i = 0; i < (1 << A); ++i) {
                if ((i >> j) & 1) continue;
                float2 &a = v[i], &b = v[i | (1 << j)];
                a.x += b.y;                    // a' = a - i b
                a.y -= b.x;
                b.x = fmaf(-2.f, b.x, -a.y);   // i a - 2b with the updated a
                b.y = fmaf(-2.f, b.y, a.x);
            }
        } else {
#pragma unroll
            for (int i = 0; i < (1 << A); ++i) {
                if ((i >> j) & 1) continue;
                float2 &a = v[i], &b = v[i | (1 << j)];
                a.x += b.x;
                a.y += b.y;
                b.x = fmaf(-2.f, b.x, a.x);
                b.y = fmaf(-2.f, b.y, a.y);
            }
        }
    }
}

// CTAs per (bin, high pattern) unit of a two-round plan: 2^(13 - c) atoms per CTA.
inline int k2_atom_groups(int K, int c) {
    const int apc = k2T >> (c - 6);
    return (K + apc - 1) / apc;
}
// Calls fn(integral_constant<C>) for a two-round plan's chunk (10, 11, 12 qubits).
template <typename Fn>
void with_chunk2(int c, Fn &&fn) {
    switch (c) {
        case 10: fn(std::integral_constant<int, 10>()); break;
        case 11: fn(std::integral_constant<int, 11>()); break;
        default: fn(std::integral_constant<int, 12>()); break;
    }
}

// Exchange A -> B: element i of thread t (= lo) goes to 66 i + t; round B
// reads elements 2 jj, 2 jj + 1 of thread t (= hi) at 66 t + 2 jj as one
// float4; the cached forward writes its round-B values back to the same
// positions (each thread overwrites only its own row).
__device__ __forceinline__ void k2_store_A(const float2 (&v)[64], float2 *wk, uint32_t t) {
#pragma unroll
    for (int i = 0; i < 64; ++i) wk[k2Row * i + t] = v[i];
}
// The same for TA = C - 6 thread bits: element i of thread t is u = t + 2^TA i.
template <int TA>
__device__ __forceinline__ void k2_store_A_g(const float2 (&v)[64], float2 *wk, uint32_t t) {
    if constexpr (TA == 6) {
        k2_store_A(v, wk, t);
    } else {
#pragma unroll
        for (int i = 0; i < 64; ++i) wk[k2Row * ((i << TA) >> 6) + ((i << TA) & 63) + t] = v[i];
    }
}
// Barrier of one atom's 2^TA threads: a named barrier of 64 (TA = 6), else
// the atom's lanes of its warp (TA <= 5: an atom lies inside one warp, and
// an inactive atom's lanes may skip the loop that waits here).
template <int TA>
__device__ __forceinline__ void k2_bar_atom_g(uint32_t ai) {
    static_assert(TA >= 4 && TA <= 6, "chunks of 10..12 qubits");
    if constexpr (TA == 6) k2_bar_atom(ai);
    else if constexpr (TA == 5) __syncwarp();
    else __syncwarp(0xffffu << (16u * (ai & 1u)));
}
__device__ __forceinline__ void k2_store_B(const float2 (&v)[64], float2 *wk, uint32_t t) {
    float4 *w4 = reinterpret_cast<float4 *>(wk + k2Row * t);
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) w4[jj] = make_float4(v[2 * jj].x, v[2 * jj].y, v[2 * jj + 1].x, v[2 * jj + 1].y);
}
__device__ __forceinline__ void k2_load_B(float2 (&v)[64], const float2 *wk, uint32_t t) {
    const float4 *w4 = reinterpret_cast<const float4 *>(wk + k2Row * t);
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
        const float4 q = w4[jj];
        v[2 * jj] = make_float2(q.x, q.y);
        v[2 * jj + 1] = make_float2(q.z, q.w);
    }
}

// Forward CTA = (bin, high pattern f, atom pair kp).  Per setting: round A,
// the exchange, round B, w_k 2^-m |.|^2 into the atom's exchange buffer (as
// floats, once every thread of the atom has read its round-B values), then
// the gather at the setting's observed outcomes in chunk f into the atom's
// slice of the partial buffer.  Without a separate float buffer a CTA needs
// 74 KB of shared memory: three CTAs (12 warps) per SM.  Per setting, one
// block barrier (the staged outcomes) and three barriers of the atom's 64
// threads (the exchange, buffer reuse before the float writes, and the
// gather before the next setting's exchange).
//
// CACHE (the evaluate path): the round-B values stay in the exchange buffer as
// complex numbers instead (each thread rewrites only its own row, which only
// it read), and the gather also stores them, unscaled, at the observed
// outcomes into the atom's slice of a.phi_obs, for the cached adjoint.
// C < 12: 2^(13-C) atoms per CTA (the "two atoms" above become that many).
template <bool CACHE, int C = 12>
__device__ __forceinline__ void forward_2r_body(const FwdArgs a, const int cta) {
    constexpr int TA = C - 6, APC = k2T >> TA;  // thread bits per atom, atoms per CTA
    constexpr K2Smem sp = k2_smem_fwd();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem + sp.stage);
    uint2 *masks_sm = reinterpret_cast<uint2 *>(smem + sp.masks);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    uint32_t *tmem_sm = reinterpret_cast<uint32_t *>(smem + sp.tmem);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, t = tid & ((1u << TA) - 1u), half = tid >> TA;
    const int KP = (a.K + APC - 1) / APC;
    const int unit = cta;
    const int kp = unit % KP;
    const int rest = unit / KP;
    const uint32_t f = rest & ((1u << a.r) - 1u);
    const int bin = rest >> a.r;
    if (bin >= *a.n_bins || (a.skip && *a.skip)) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    const int k = APC * kp + (int)half;
    const bool active = k < a.K;
    float2 *wk = reinterpret_cast<float2 *>(smem + sp.work) + half * (k2Row << TA);
    float *pb = reinterpret_cast<float *>(wk);  // w |.|^2 at k2_fpos(u), after the exchange
    constexpr uint32_t cmask = (1u << C) - 1u;
    if (warp == 0) tm_alloc(tmem_sm, k2ColsFwd);
    fx_stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, masks_sm, meta_sm);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t t_src = tmem_sm[0] + ((warp * 32u) << 16);
    const int bcount = b.count;
    const uint32_t *outcome = a.outcome;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            uint32_t *dst = stage + (si & 1) * k2Stage;
            const int nst = mt.cnt < k2Stage ? mt.cnt : k2Stage;
            for (int j = tid; j < nst; j += k2T) cp_async4(dst + j, outcome + mt.lo + j);
        }
        cp_async_commit();
    };
    const float wkk = active ? a.w[k] : 0.f;
    float *pk = a.ppart + (size_t)(active ? k : 0) * a.nnz;
    // the CTA's atoms' weights (the small-atom gather serves every atom)
    float wsm[TA < 6 ? APC : 1];
#pragma unroll
    for (int aa = 0; aa < (TA < 6 ? APC : 1); ++aa) wsm[aa] = APC * kp + aa < a.K ? a.w[APC * kp + aa] : 0.f;
    issue(0);
    k2_build_source<C>(t_src, a.psi + (size_t)bin * a.src_bin_stride + (size_t)(active ? k : 0) * D, active, f,
                       b.xytop, b.ytop, t);
    tm_wait_st();
    for (int si = 0; si < bcount; ++si) {
        const uint2 mk = masks_sm[si];
        const SetMeta mt = meta_sm[si];
        float2 v[64];
        k2_tm_ld64(t_src, v);
        // rounds A (R = 0) and B (R = 1) share one butterfly site: a 6-bit
        // round unrolled twice does not fit the instruction cache
#pragma unroll 1
        for (int R = 0; R < 2; ++R) {
            // round A: chunk bits 6..C-1 (its register bits 6-TA..5), round B: bits 0..5
            const uint32_t sh = R ? 0u : (uint32_t)TA, keep = R ? 63u : 63u & ~((1u << (6 - TA)) - 1u);
            butterfly_herm<6>(v, (mk.x >> sh) & keep, (mk.y >> sh) & keep);
            if (R == 0) {
                k2_store_A_g<TA>(v, wk, t);
                k2_bar_atom_g<TA>(half);
                k2_load_B(v, wk, t);
            }
        }
        const float sc = wkk * mt.cs;
        if (CACHE) {
            k2_store_B(v, wk, t);
        } else {
            k2_bar_atom_g<TA>(half);  // every round-B read of the exchange buffer is done
            float4 *p4 = reinterpret_cast<float4 *>(pb + k2FRow * t);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                float4 o;
                o.x = scaled_abs2(sc, v[4 * q]);
                o.y = scaled_abs2(sc, v[4 * q + 1]);
                o.z = scaled_abs2(sc, v[4 * q + 2]);
                o.w = scaled_abs2(sc, v[4 * q + 3]);
                p4[q] = o;
            }
        }
        cp_async_wait0();
        __syncthreads();  // this setting's stage landed (every thread's copies); the floats are written
        // the stage buffer of setting si + 1 was last read by the gather of si - 1,
        // which every thread finished before the barrier above
        issue(si + 1);
        const uint32_t *st = stage + (si & 1) * k2Stage;
        if constexpr (TA < 6) {
            // Small atoms (2^TA threads) would each walk the setting's whole
            // outcome list; instead every thread reads an outcome once and
            // serves all of the CTA's atoms (block barriers around the gather).
            float2 *W = reinterpret_cast<float2 *>(smem + sp.work);
            for (int j = tid; j < mt.cnt; j += k2T) {
                const uint32_t u = (j < k2Stage ? st[j] : outcome[mt.lo + j]) & cmask;
#pragma unroll
                for (int aa = 0; aa < APC; ++aa) {
                    const int ka = APC * kp + aa;
                    if (ka >= a.K) break;
                    const float2 *wa = W + aa * (k2Row << TA);
                    float *pa = a.ppart + (size_t)ka * a.nnz;
                    if (CACHE) {
                        const float2 ph = wa[k2Row * (u >> 6) + (u & 63u)];
                        pa[mt.lo + j] = scaled_abs2(wsm[aa] * mt.cs, ph);
                        a.phi_obs[(size_t)ka * a.nnz + mt.lo + j] = ph;
                    } else {
                        pa[mt.lo + j] = reinterpret_cast<const float *>(wa)[k2_fpos(u)];
                    }
                }
            }
            if (a.p_dense) {
                const int s = a.order[b.start + si];
                float *pd = a.p_dense + (size_t)s * D + ((size_t)f << C);
                for (uint32_t u = tid; u <= cmask; u += k2T) {
#pragma unroll
                    for (int aa = 0; aa < APC; ++aa) {
                        if (APC * kp + aa >= a.K) break;
                        const float2 *wa = W + aa * (k2Row << TA);
                        atomicAdd(pd + u, CACHE ? scaled_abs2(wsm[aa] * mt.cs, wa[k2Row * (u >> 6) + (u & 63u)])
                                                : reinterpret_cast<const float *>(wa)[k2_fpos(u)]);
                    }
                }
            }
            __syncthreads();  // the gather is done before the next setting's exchange stores
            continue;
        }
        if (active && CACHE) {
            float2 *phk = a.phi_obs + (size_t)k * a.nnz;
            for (int j = t; j < mt.cnt; j += (1 << TA)) {
                const uint32_t u = (j < k2Stage ? st[j] : outcome[mt.lo + j]) & cmask;
                const float2 ph = wk[k2Row * (u >> 6) + (u & 63u)];
                pk[mt.lo + j] = scaled_abs2(sc, ph);
                phk[mt.lo + j] = ph;
            }
            if (a.p_dense) {
                const int s = a.order[b.start + si];
                float *pd = a.p_dense + (size_t)s * D + ((size_t)f << C);
                for (uint32_t u = t; u <= cmask; u += (1u << TA)) {
                    const float2 ph = wk[k2Row * (u >> 6) + (u & 63u)];
                    atomicAdd(pd + u, scaled_abs2(sc, ph));
                }
            }
        } else if (active) {
            for (int j = t; j < mt.cnt; j += (1 << TA)) {
                const uint32_t u = (j < k2Stage ? st[j] : outcome[mt.lo + j]) & cmask;
                pk[mt.lo + j] = pb[k2_fpos(u)];
            }
            if (a.p_dense) {
                const int s = a.order[b.start + si];
                float *pd = a.p_dense + (size_t)s * D + ((size_t)f << C);
                for (uint32_t u = t; u <= cmask; u += (1u << TA)) atomicAdd(pd + u, pb[k2_fpos(u)]);
            }
        }
        k2_bar_atom_g<TA>(half);  // the gather is done before the next setting's exchange stores
    }
    cp_async_wait0();
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(tmem_sm[0], k2ColsFwd);
    }
}
template <bool CACHE, int C = 12>
__global__ void __launch_bounds__(k2T, 3) k_forward_2r(const FwdArgs a) {
    forward_2r_body<CACHE, C>(a, blockIdx.x);
}
template <bool CACHE, int C = 12>
__global__ void __launch_bounds__(k2T, 3) k_forward_2r_multi(const FwdArgs *__restrict__ args, const int *__restrict__ start, int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const FwdArgs a = args[i];
    forward_2r_body<CACHE, C>(a, (int)blockIdx.x - start[i]);
}

