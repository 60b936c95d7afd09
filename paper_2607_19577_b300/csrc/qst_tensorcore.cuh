// Tensor-core chunk kernels (plan precision 1..3; included inside qst.cu's
// anonymous namespace, after qst_tworound_packed.cuh).
//
// The 12-qubit chunk transform of a setting (the grouped form of the rotation
// U_s psi_k, Eq. atom-response, with qubits grouped six at a time) as two
// dense group products on the tcgen05 tensor cores.  A chunk is the 64 x 64
// array X[hi][lo] (u = lo + 64 hi); with the Hermitian chunk factors of
// qst_tworound.cuh, H = H_hi (x) H_lo (entries 0, +-1, +-i before the
// 2^-m/2 scale, so exact in BF16),
//
//   step 1:  T[hi'][lo] = sum_hi H_hi[hi'][hi] X[hi][lo]     (rows lo, K = hi)
//   step 2:  P[hi][lo'] = sum_lo H_lo[lo'][lo] T[hi][lo]     (rows hi, K = lo)
//
// Both are right products x G of row vectors with a complex 64 x 64 G = H^T,
// written as real 128 x 128 products over interleaved (index, re/im) pairs:
// A = the data rows (M = 128: two atoms of 64 rows), B = the real form of G
// (N = 128), K = 128, D in TMEM in FP32.  The data are split into T BF16
// terms x = x1 + x2 + ... (x1 = bf16(x), x2 = bf16(x - x1), ...), each term
// multiplied by the exact operator, FP32 accumulation: T = 3 carries all 24
// bits of an FP32 value, T = 1 is plain BF16.  Because the chunk factors are
// Hermitian the adjoint's inverse transform is the same pair of products in
// the other order (lo first), with the same operators.
//
// Operators: the real form of G for each of the 3^6 basis patterns of a
// six-qubit group, built once per plan (k_tc_ops, 729 x 32 KB, stays in L2),
// laid out as the MMA's B operand (no swizzle, K-major core matrices: 8 rows
// x 16 bytes, K-adjacent core matrices 2048 bytes apart, 8-row groups 128
// bytes apart), so one bulk copy per setting and group lands it in shared
// memory.  Data operand (A): same core matrices, 8-row groups 128 bytes
// apart, K-adjacent core matrices kTcLBO = 2064 bytes apart: the 16 bytes of
// padding put the 4-byte stores of 32 consecutive K positions (one row) into
// 32 distinct banks.
//
// CTA = (bin, high pattern f, atom pair), 16 warps.  Warp w reaches TMEM
// lanes 32 (w % 4) .. + 31 (its rows) and handles columns 32 (w / 4) .. + 31
// (16 complex values of each row).  Per setting: the source (TMEM, FP32, built
// once per unit as in the two-round kernels) is split into the A terms; one
// thread issues step 1's 8 T MMAs and commits them to an mbarrier; the D rows
// are split into the A terms of step 2 (the transpose between the steps);
// step 2; the epilogue reads D.  The next setting's operators are copied in
// as soon as the MMAs that read the previous ones have completed.  Every wait
// on an mbarrier is bounded: past the limit the kernel sets QST_DEV_TIMEOUT in
// the status word, stops issuing work, waits (bounded) for its own copies in
// flight, frees its TMEM and returns.

constexpr int kTcT = 512;               // threads per CTA (16 warps)
constexpr uint32_t kTcLBO = 2064;       // A operand: bytes between K-adjacent core matrices
constexpr uint32_t kTcASz = 33024;      // bytes of one A term (15 kTcLBO + 2048, rounded up)
constexpr uint32_t kTcOpLBO = 2048;     // B operand (operator): bytes between K-adjacent core matrices
constexpr uint32_t kTcOpBytes = 32768;  // one operator (128 x 128 BF16)
constexpr int kTcOps = 729;             // 3^6 basis patterns of a six-qubit group
constexpr uint32_t kTcCols = 256;       // TMEM columns: 0..127 source / accumulator, 128..255 D
constexpr int kTcSpin = 1 << 22;        // try_wait polls before a wait is abandoned
constexpr int kTcStage = 512;           // observed entries per setting staged by cp.async
// instruction descriptor, kind::f16: FP32 D (bits 4-5 = 1), BF16 A and B
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
static_assert(15 * kTcLBO + 2048 <= kTcASz && kTcASz % 128 == 0, "A term size");

struct TcSmem {
    int ops, work, stage, masks, meta, bar, flag, tmem, total;
};
// work: the T A terms, aliased by the epilogue buffers (forward: w |.|^2 as
// floats, or the complex transforms for the cache); stage: the forward's
// outcome indices, or the adjoint's (outcome, c, transform) per atom.
template <int T, bool ADJ, bool CACHE>
__host__ __device__ constexpr TcSmem tc_smem() {
    TcSmem sp{};
    sp.ops = 0;
    sp.work = sp.ops + 2 * (int)kTcOpBytes;
    const int a_bytes = T * (int)kTcASz;
    const int e_bytes = ADJ ? 0 : (CACHE ? 2 * k2Buf * 8 : 2 * k2FBuf * 4);
    sp.stage = sp.work + (a_bytes > e_bytes ? a_bytes : e_bytes);
    const int st_bytes = ADJ ? 2 * 2 * kTcStage * (4 + 4 + 8) : 2 * kTcStage * 4;
    sp.masks = sp.stage + st_bytes;
    sp.meta = sp.masks + kMaxBin * (int)sizeof(uint2);
    sp.bar = sp.meta + kMaxBin * (int)sizeof(SetMeta);
    sp.flag = sp.bar + 3 * 8;
    sp.tmem = sp.flag + 8;
    sp.total = sp.tmem + 16;
    return sp;
}
// Every tensor-core CTA takes the whole opt-in shared memory (one CTA per SM
// either way: 512 threads at up to 120 registers), so every address an MMA
// descriptor can reach, under either reading of its two strides, lies inside
// the CTA's own allocation.
constexpr int kTcSmemAlloc = 227 * 1024;
static_assert(tc_smem<3, true, false>().total <= kTcSmemAlloc, "adjoint shared memory");
static_assert(tc_smem<3, false, true>().total <= kTcSmemAlloc, "forward shared memory");
static_assert(2 * (int)kTcOpBytes + 2 * (int)kTcASz + 14 * (int)kTcLBO + 128 + 15 * (int)kTcLBO + 128 <= kTcSmemAlloc,
              "A reads of the last term stay inside the allocation with LBO and SBO exchanged");
static_assert(2 * (int)kTcOpBytes + 14 * (int)kTcOpLBO + 128 + 15 * (int)kTcOpLBO + 128 <= kTcSmemAlloc,
              "B reads of slot 1 stay inside the allocation with LBO and SBO exchanged");
static_assert(tc_smem<1, false, true>().stage % 16 == 0 && tc_smem<3, true, false>().bar % 8 == 0, "alignment");

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo) {
    // start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO = 128 >> 4 (32-45), version 1 at bit 46, no swizzle
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) | ((uint64_t)(128u >> 4) << 32) |
           (1ull << 46);
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mb_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mb_wait(uint32_t bar, uint32_t parity) {
    for (int i = 0; i < kTcSpin; ++i) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.u32 %0, 1, 0, P;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// one operator (32 KB, contiguous in the table) into a B slot, completing on bar
__device__ __forceinline__ void tc_load_op(uint32_t dst, const unsigned char *src, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kTcOpBytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(kTcOpBytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void st_sh_b32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void st_sh_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
// (re, im) -> one word: re's BF16 in the low half (the lower K index), im's in the high half
__device__ __forceinline__ uint32_t bf16x2(float re, float im) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(im), "f"(re));
    return d;
}
// Split 16 complex values (32 words, re/im interleaved) into T BF16 terms,
// largest first; every residual x - bf16(x) is exact in FP32.
template <int T>
__device__ __forceinline__ void tc_split(const uint32_t (&r)[32], uint32_t (&h)[T][16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float re = __uint_as_float(r[2 * i]), im = __uint_as_float(r[2 * i + 1]);
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint32_t w = bf16x2(re, im);
            h[t][i] = w;
            if (t + 1 < T) {
                re -= __uint_as_float(w << 16);
                im -= __uint_as_float(w & 0xFFFF0000u);
            }
        }
    }
}
// Base-3 index of a six-qubit group's bases (0 = Z, 1 = X, 2 = Y per qubit).
__device__ __forceinline__ uint32_t tc_code(uint32_t xy6, uint32_t y6) {
    uint32_t idx = 0, p3 = 1;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        idx += (((xy6 >> q) & 1u) ? (((y6 >> q) & 1u) ? 2u : 1u) : 0u) * p3;
        p3 *= 3u;
    }
    return idx;
}
// Issue step's 8 T MMAs (terms smallest first, K in steps of 16) and commit
// them to bar.  accumulate: add to D's previous contents from the first MMA on.
template <int T>
__device__ __forceinline__ void tc_issue(uint32_t d_tmem, uint32_t a_base, uint32_t b_base, uint32_t accumulate,
                                         uint32_t bar) {
    uint32_t acc = accumulate;
#pragma unroll
    for (int t = T - 1; t >= 0; --t) {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            tc_mma(d_tmem, tc_desc(a_base + (uint32_t)t * kTcASz + 2u * kTcLBO * kk, kTcLBO),
                   tc_desc(b_base + 2u * kTcOpLBO * kk, kTcOpLBO), acc);
            acc = 1u;
        }
    }
    tc_commit(bar);
}

// The real form of G = H^T for every basis pattern of a six-qubit group, in
// the B operand's layout: element (n, k), n = 2 l + re/im of the output
// index l, k = 2 j + re/im of the input index j, holds the coefficient of
// x_k in (x G)_n.  H[l][j] = prod_q h_q[l_q][j_q] with h_Z = I,
// h_X = [[1,1],[1,-1]], h_Y = [[1,-i],[i,-1]] (the chunk factors of the
// two-round kernels).
__global__ void k_tc_ops(unsigned short *tab) {
    const uint32_t idx = blockIdx.x;
    uint32_t code[6], rest = idx;
    for (int q = 0; q < 6; ++q) {
        code[q] = rest % 3u;
        rest /= 3u;
    }
    unsigned short *o = tab + (size_t)idx * (kTcOpBytes / 2);
    for (uint32_t e = threadIdx.x; e < 128u * 128u; e += blockDim.x) {
        const uint32_t n = e >> 7, k = e & 127u, l = n >> 1, j = k >> 1;
        bool zero = false;
        uint32_t ph = 0;  // H[l][j] = i^ph
        for (int q = 0; q < 6; ++q) {
            const uint32_t lb = (l >> q) & 1u, jb = (j >> q) & 1u;
            if (code[q] == 0) {
                if (lb != jb) zero = true;
            } else if (code[q] == 1) {
                if (lb & jb) ph += 2;
            } else {
                ph += lb ? (jb ? 2u : 1u) : (jb ? 3u : 0u);
            }
        }
        int gr = 0, gi = 0;  // G[j][l] = H[l][j]
        if (!zero) {
            gr = (ph & 3u) == 0 ? 1 : ((ph & 3u) == 2 ? -1 : 0);
            gi = (ph & 3u) == 1 ? 1 : ((ph & 3u) == 3 ? -1 : 0);
        }
        const uint32_t co = n & 1u, ci = k & 1u;
        const int v = co == 0 ? (ci == 0 ? gr : -gi) : (ci == 0 ? gi : gr);
        const uint32_t byte = (k >> 3) * kTcOpLBO + (n >> 3) * 128u + (n & 7u) * 16u + (k & 7u) * 2u;
        o[byte >> 1] = v == 0 ? (unsigned short)0 : (v > 0 ? (unsigned short)0x3F80 : (unsigned short)0xBF80);
    }
}

// Per-CTA control of the tensor-core kernels: barriers, phases, operator
// copies in flight (thread 0's view) and the abort flag.
struct TcCtl {
    uint32_t bar_op[2], bar_mma;
    uint32_t ph_op[2], ph_mma;
    bool inflight[2];
    volatile int *abort_sm;
    int *status;
    __device__ void fail() {
        *abort_sm = 1;
        if (status) atomicOr(status, QST_DEV_TIMEOUT);
    }
    // thread 0: wait for the operator in slot s, then issue the step and commit
    template <int T>
    __device__ void step(uint32_t d_tmem, uint32_t a_base, uint32_t b_base, int s, uint32_t accumulate) {
        tm_fence_after();
        if (mb_wait(bar_op[s], ph_op[s])) {
            inflight[s] = false;
            ph_op[s] ^= 1u;
            tc_issue<T>(d_tmem, a_base, b_base, accumulate, bar_mma);
        } else {
            fail();
            tc_commit(bar_mma);  // nothing issued: the commit keeps the other threads' wait short
        }
    }
    // every thread: wait for the committed MMAs (the phases advance in lockstep)
    __device__ void wait_mma() {
        if (!mb_wait(bar_mma, ph_mma)) fail();
        ph_mma ^= 1u;
        tm_fence_after();
    }
    __device__ void load(int s, uint32_t dst, const unsigned char *src) {
        tc_load_op(dst, src, bar_op[s]);
        inflight[s] = true;
    }
    // thread 0 on the way out: copies still in flight land before the CTA exits
    __device__ void drain() {
        for (int s = 0; s < 2; ++s)
            if (inflight[s]) {
                if (!mb_wait(bar_op[s], ph_op[s])) fail();
                inflight[s] = false;
            }
    }
};

// Source rows -> A terms: this thread's lane (row) and column quarter cq hold
// 16 complex values at K pairs 16 cq .. 16 cq + 15; four 16-byte stores per term.
template <int T>
__device__ __forceinline__ void tc_store_rows(const uint32_t (&r)[32], uint32_t a_base, uint32_t row, uint32_t cq) {
    uint32_t h[T][16];
    tc_split<T>(r, h);
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            st_sh_v4(a_base + (uint32_t)t * kTcASz + (4u * cq + j) * kTcLBO + row * 16u, h[t][4 * j], h[t][4 * j + 1],
                     h[t][4 * j + 2], h[t][4 * j + 3]);
}
// D rows -> A terms of the next step, transposed within the atom: this
// thread's row is (atom, x) and its 16 values are y = 16 cq + i; they go to
// row (atom, y) at K pair x, one 4-byte store per value and term.
template <int T>
__device__ __forceinline__ void tc_store_transposed(const uint32_t (&r)[32], uint32_t a_base, uint32_t atom,
                                                    uint32_t x, uint32_t cq) {
    uint32_t h[T][16];
    tc_split<T>(r, h);
    const uint32_t base = a_base + (x >> 2) * kTcLBO + (x & 3u) * 4u + (64u * atom + 16u * cq) * 16u;
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int i = 0; i < 16; ++i) st_sh_b32(base + (uint32_t)t * kTcASz + 16u * i, h[t][i]);
}

// Forward, tensor cores.  Same unit as k_forward_2r; per setting the
// |.|^2 weighting and the gather at the observed outcomes (and, with CACHE,
// the store of the transforms) follow the two-round kernel.
template <int T, bool CACHE>
__global__ void __launch_bounds__(kTcT, 1) k_forward_tc(const FwdArgs a) {
    constexpr TcSmem sp = tc_smem<T, false, CACHE>();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem + sp.stage);
    uint2 *masks_sm = reinterpret_cast<uint2 *>(smem + sp.masks);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    uint32_t *tmem_sm = reinterpret_cast<uint32_t *>(smem + sp.tmem);
    volatile int *abort_sm = reinterpret_cast<volatile int *>(smem + sp.flag);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t cq = warp >> 2, row = 32u * (warp & 3u) + lane, atom = row >> 6, x = row & 63u;
    const int KP = (a.K + 1) >> 1;
    const int unit = blockIdx.x;
    const int kp = unit % KP;
    const int rest = unit / KP;
    const uint32_t f = rest & ((1u << a.r) - 1u);
    const int bin = rest >> a.r;
    if (bin >= *a.n_bins || (a.skip && *a.skip)) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    const int ka = 2 * kp + (int)(tid >> 8);  // the atom of this thread's gather half
    const bool active_g = ka < a.K;
    constexpr uint32_t cmask = 4095u;
    const uint32_t s_ops = smem_u32(smem + sp.ops), s_work = smem_u32(smem + sp.work);
    TcCtl ctl;
    ctl.bar_op[0] = smem_u32(smem + sp.bar);
    ctl.bar_op[1] = ctl.bar_op[0] + 8u;
    ctl.bar_mma = ctl.bar_op[0] + 16u;
    ctl.ph_op[0] = ctl.ph_op[1] = ctl.ph_mma = 0u;
    ctl.inflight[0] = ctl.inflight[1] = false;
    ctl.abort_sm = abort_sm;
    ctl.status = a.status;
    if (warp == 0) tm_alloc(tmem_sm, kTcCols);
    if (tid == 0) {
        mb_init(ctl.bar_op[0]);
        mb_init(ctl.bar_op[1]);
        mb_init(ctl.bar_mma);
        *abort_sm = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fx_stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, masks_sm, meta_sm);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const int bcount = b.count;
    const unsigned char *ops = a.tc_ops;
    if (tid == 0 && bcount > 0) {
        const uint2 mk = masks_sm[0];
        ctl.load(0, s_ops, ops + (size_t)tc_code((mk.x >> 6) & 63u, (mk.y >> 6) & 63u) * kTcOpBytes);
        ctl.load(1, s_ops + kTcOpBytes, ops + (size_t)tc_code(mk.x & 63u, mk.y & 63u) * kTcOpBytes);
    }
    const uint32_t tbase = tmem_sm[0];
    const uint32_t t_lane = tbase + ((32u * (warp & 3u)) << 16);
    const uint32_t t_src = t_lane + 32u * cq, t_d = t_lane + 128u + 32u * cq;
    if (tid < 128) {  // the source of atom 2 kp + tid / 64 in lanes 0..127, columns 0..127
        const int k0 = 2 * kp + (int)(tid >> 6);
        const bool act = k0 < a.K;
        k2_build_source(tbase + ((32u * warp) << 16), a.psi + (size_t)bin * a.src_bin_stride + (size_t)(act ? k0 : 0) * D,
                        act, f, b.xytop, b.ytop, tid & 63u);
        tm_wait_st();
    }
    const uint32_t *outcome = a.outcome;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            uint32_t *dst = stage + (si & 1) * kTcStage;
            const int nst = mt.cnt < kTcStage ? mt.cnt : kTcStage;
            for (int j = tid; j < nst; j += kTcT) cp_async4(dst + j, outcome + mt.lo + j);
        }
        cp_async_commit();
    };
    const float wkk = active_g ? a.w[ka] : 0.f;
    float *pk = a.ppart + (size_t)(active_g ? ka : 0) * a.nnz;
    float2 *wk = reinterpret_cast<float2 *>(smem + sp.work) + (tid >> 8) * k2Buf;  // CACHE: transforms, 66 hi + lo
    float *pb = reinterpret_cast<float *>(smem + sp.work) + (tid >> 8) * k2FBuf;   // w |.|^2 at k2_fpos(u)
    float2 *wk_row = reinterpret_cast<float2 *>(smem + sp.work) + atom * k2Buf;
    float *pb_row = reinterpret_cast<float *>(smem + sp.work) + atom * k2FBuf;
    issue(0);
    tm_fence_before();
    __syncthreads();  // the source is in TMEM
    tm_fence_after();
    const uint32_t jt = tid & 255u;
    for (int si = 0; si < bcount; ++si) {
        const SetMeta mt = meta_sm[si];
        {  // step 1's A: the source rows (atom, lo), K = (hi, re/im)
            uint32_t r[32];
            tm_ld_issue(t_src, r);
            tm_ld_wait(r);
            tc_store_rows<T>(r, s_work, row, cq);
        }
        fence_async_smem();
        tm_fence_before();
        __syncthreads();
        if (*abort_sm) break;
        if (tid == 0) ctl.step<T>(tbase + 128u, s_work, s_ops, 0, 0u);
        ctl.wait_mma();
        if (tid == 0 && si + 1 < bcount) {
            const uint2 mn = masks_sm[si + 1];
            ctl.load(0, s_ops, ops + (size_t)tc_code((mn.x >> 6) & 63u, (mn.y >> 6) & 63u) * kTcOpBytes);
        }
        {  // T rows (atom, lo) -> step 2's A rows (atom, hi), K = (lo, re/im)
            uint32_t r[32];
            tm_ld_issue(t_d, r);
            tm_ld_wait(r);
            tc_store_transposed<T>(r, s_work, atom, x, cq);
        }
        fence_async_smem();
        tm_fence_before();
        __syncthreads();
        if (*abort_sm) break;
        if (tid == 0) ctl.step<T>(tbase + 128u, s_work, s_ops + kTcOpBytes, 1, 0u);
        ctl.wait_mma();
        if (tid == 0 && si + 1 < bcount) {
            const uint2 mn = masks_sm[si + 1];
            ctl.load(1, s_ops + kTcOpBytes, ops + (size_t)tc_code(mn.x & 63u, mn.y & 63u) * kTcOpBytes);
        }
        const float sc = (2 * kp + (int)atom < a.K ? a.w[2 * kp + atom] : 0.f) * mt.cs;
        {  // the transform rows (atom, hi), lo = 16 cq + i
            uint32_t r[32];
            tm_ld_issue(t_d, r);
            tm_ld_wait(r);
            if (CACHE) {
                float4 *w4 = reinterpret_cast<float4 *>(wk_row + k2Row * x + 16u * cq);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    w4[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                        __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
            } else {
                float4 *p4 = reinterpret_cast<float4 *>(pb_row + k2FRow * x + 16u * cq);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float o[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float re = __uint_as_float(r[8 * q + 2 * e]), im = __uint_as_float(r[8 * q + 2 * e + 1]);
                        o[e] = sc * (re * re + im * im);
                    }
                    p4[q] = make_float4(o[0], o[1], o[2], o[3]);
                }
            }
        }
        tm_fence_before();
        cp_async_wait0();
        __syncthreads();  // this setting's stage landed; the epilogue buffers are written
        issue(si + 1);
        const uint32_t *st = stage + (si & 1) * kTcStage;
        const float scg = wkk * mt.cs;
        if (active_g && CACHE) {
            float2 *phk = a.phi_obs + (size_t)ka * a.nnz;
            for (int j = jt; j < mt.cnt; j += 256) {
                const uint32_t u = (j < kTcStage ? st[j] : outcome[mt.lo + j]) & cmask;
                const float2 ph = wk[k2Row * (u >> 6) + (u & 63u)];
                pk[mt.lo + j] = scg * (ph.x * ph.x + ph.y * ph.y);
                phk[mt.lo + j] = ph;
            }
            if (a.p_dense) {
                const int s = a.order[b.start + si];
                float *pd = a.p_dense + (size_t)s * D + ((size_t)f << 12);
                for (uint32_t u = jt; u <= cmask; u += 256) {
                    const float2 ph = wk[k2Row * (u >> 6) + (u & 63u)];
                    atomicAdd(pd + u, scg * (ph.x * ph.x + ph.y * ph.y));
                }
            }
        } else if (active_g) {
            for (int j = jt; j < mt.cnt; j += 256) {
                const uint32_t u = (j < kTcStage ? st[j] : outcome[mt.lo + j]) & cmask;
                pk[mt.lo + j] = pb[k2_fpos(u)];
            }
            if (a.p_dense) {
                const int s = a.order[b.start + si];
                float *pd = a.p_dense + (size_t)s * D + ((size_t)f << 12);
                for (uint32_t u = jt; u <= cmask; u += 256) atomicAdd(pd + u, pb[k2_fpos(u)]);
            }
        }
        __syncthreads();  // the gather is done before the next setting's A terms overwrite the buffers
    }
    cp_async_wait0();
    if (tid == 0) ctl.drain();
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(tbase, kTcCols);
    }
}

// Adjoint from the stored transforms, tensor cores.  Same unit as
// k_adjoint_2c.  Per setting: the dense y = c 2^-m phi at the observed
// outcomes of chunk f (zero elsewhere) as step 1's A rows (atom, hi), K =
// (lo, re/im); step 1 with the lo operator; the transpose into rows (atom,
// lo); step 2 with the hi operator accumulates into the unit's accumulator
// (TMEM columns 0..127), which is written to the z buffer at the end.
template <int T>
__global__ void __launch_bounds__(kTcT, 1) k_adjoint_tc(const AdjArgs a) {
    if (a.skip && *a.skip) return;
    constexpr TcSmem sp = tc_smem<T, true, false>();
    extern __shared__ __align__(16) unsigned char smem[];
    uint2 *masks_sm = reinterpret_cast<uint2 *>(smem + sp.masks);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    uint32_t *tmem_sm = reinterpret_cast<uint32_t *>(smem + sp.tmem);
    volatile int *abort_sm = reinterpret_cast<volatile int *>(smem + sp.flag);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t cq = warp >> 2, row = 32u * (warp & 3u) + lane, atom = row >> 6, x = row & 63u;
    const int KP = (a.K + 1) >> 1;
    const int unit = blockIdx.x;
    const int kp = unit % KP;
    const int rest = unit / KP;
    const uint32_t f = rest & ((1u << a.r) - 1u);
    const int bin = rest >> a.r;
    if (bin >= *a.n_bins) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    const uint32_t half = tid >> 8, jt = tid & 255u;
    const int ks = 2 * kp + (int)half;  // the atom of this thread's scatter half
    const bool active_s = ks < a.K;
    constexpr uint32_t cmask = 4095u;
    const uint32_t s_ops = smem_u32(smem + sp.ops), s_work = smem_u32(smem + sp.work);
    uint32_t *stu = reinterpret_cast<uint32_t *>(smem + sp.stage) + half * 2 * kTcStage;
    float *stc = reinterpret_cast<float *>(smem + sp.stage + 2 * 2 * kTcStage * 4) + half * 2 * kTcStage;
    float2 *stp = reinterpret_cast<float2 *>(smem + sp.stage + 2 * 2 * kTcStage * 8) + half * 2 * kTcStage;
    TcCtl ctl;
    ctl.bar_op[0] = smem_u32(smem + sp.bar);
    ctl.bar_op[1] = ctl.bar_op[0] + 8u;
    ctl.bar_mma = ctl.bar_op[0] + 16u;
    ctl.ph_op[0] = ctl.ph_op[1] = ctl.ph_mma = 0u;
    ctl.inflight[0] = ctl.inflight[1] = false;
    ctl.abort_sm = abort_sm;
    ctl.status = a.status;
    if (warp == 0) tm_alloc(tmem_sm, kTcCols);
    if (tid == 0) {
        mb_init(ctl.bar_op[0]);
        mb_init(ctl.bar_op[1]);
        mb_init(ctl.bar_mma);
        *abort_sm = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fx_stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, masks_sm, meta_sm);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const int bcount = b.count;
    const unsigned char *ops = a.tc_ops;
    if (tid == 0 && bcount > 0) {
        const uint2 mk = masks_sm[0];
        ctl.load(0, s_ops, ops + (size_t)tc_code(mk.x & 63u, mk.y & 63u) * kTcOpBytes);
        ctl.load(1, s_ops + kTcOpBytes, ops + (size_t)tc_code((mk.x >> 6) & 63u, (mk.y >> 6) & 63u) * kTcOpBytes);
    }
    const uint32_t tbase = tmem_sm[0];
    const uint32_t t_lane = tbase + ((32u * (warp & 3u)) << 16);
    const uint32_t t_acc = t_lane + 32u * cq, t_d = t_lane + 128u + 32u * cq;
    {
        uint32_t z[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) z[i] = 0u;
        tm_st(t_acc, z);
        tm_wait_st();
    }
    const uint32_t *outcome = a.outcome;
    const float *c_obs = a.c_obs;
    const float2 *phk = a.phi_obs + (size_t)(active_s ? ks : 0) * a.nnz;
    auto issue = [&](int si) {
        if (si < bcount && active_s) {
            const SetMeta mt = meta_sm[si];
            const int nst = mt.cnt < kTcStage ? mt.cnt : kTcStage;
            const int o = (si & 1) * kTcStage;
            for (int j = jt; j < nst; j += 256) {
                cp_async4(stu + o + j, outcome + mt.lo + j);
                cp_async4(stc + o + j, c_obs + mt.lo + j);
                cp_async8(stp + o + j, phk + mt.lo + j);
            }
        }
        cp_async_commit();
    };
    issue(0);
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    for (int si = 0; si < bcount; ++si) {
        const SetMeta mt = meta_sm[si];
        for (uint32_t o = tid * 16u; o < (uint32_t)T * kTcASz; o += kTcT * 16u)
            st_sh_v4(s_work + o, zero4.x, zero4.y, zero4.z, zero4.w);
        cp_async_wait0();  // this thread's entries of setting si have landed
        __syncthreads();   // the zeros are written
        issue(si + 1);     // into the buffer this thread read for setting si - 1
        if (active_s) {
            const int o = (si & 1) * kTcStage;
            const uint32_t base = s_work + 64u * 16u * half;
            for (int j = jt; j < mt.cnt; j += 256) {
                const bool st = j < kTcStage;
                const uint32_t u = (st ? stu[o + j] : outcome[mt.lo + j]) & cmask;
                const float cy = (st ? stc[o + j] : c_obs[mt.lo + j]) * mt.cs;
                const float2 ph = st ? stp[o + j] : phk[mt.lo + j];
                float re = cy * ph.x, im = cy * ph.y;
                const uint32_t lo = u & 63u, hi = u >> 6;
                const uint32_t addr = base + (lo >> 2) * kTcLBO + (lo & 3u) * 4u + hi * 16u;
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const uint32_t w = bf16x2(re, im);
                    st_sh_b32(addr + (uint32_t)t * kTcASz, w);
                    if (t + 1 < T) {
                        re -= __uint_as_float(w << 16);
                        im -= __uint_as_float(w & 0xFFFF0000u);
                    }
                }
            }
        }
        fence_async_smem();
        tm_fence_before();
        __syncthreads();
        if (*abort_sm) break;
        if (tid == 0) ctl.step<T>(tbase + 128u, s_work, s_ops, 0, 0u);
        ctl.wait_mma();
        if (tid == 0 && si + 1 < bcount) {
            const uint2 mn = masks_sm[si + 1];
            ctl.load(0, s_ops, ops + (size_t)tc_code(mn.x & 63u, mn.y & 63u) * kTcOpBytes);
        }
        {  // rows (atom, hi) -> step 2's A rows (atom, lo), K = (hi, re/im)
            uint32_t r[32];
            tm_ld_issue(t_d, r);
            tm_ld_wait(r);
            tc_store_transposed<T>(r, s_work, atom, x, cq);
        }
        fence_async_smem();
        tm_fence_before();
        __syncthreads();
        if (*abort_sm) break;
        if (tid == 0) ctl.step<T>(tbase, s_work, s_ops + kTcOpBytes, 1, 1u);
        ctl.wait_mma();
        if (tid == 0 && si + 1 < bcount) {
            const uint2 mn = masks_sm[si + 1];
            ctl.load(1, s_ops + kTcOpBytes, ops + (size_t)tc_code((mn.x >> 6) & 63u, (mn.y >> 6) & 63u) * kTcOpBytes);
        }
        // each thread has seen step 2 complete (its own wait) before it zeroes the A terms
    }
    cp_async_wait0();
    if (tid == 0) ctl.drain();
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (2 * kp + (int)atom < a.K && !*abort_sm) {
        uint32_t r[32];
        tm_ld_issue(t_acc, r);
        tm_ld_wait(r);
        float2 *zo = a.zbuf + ((size_t)bin * a.K + (2 * kp + atom)) * D + ((size_t)f << 12) + x;
#pragma unroll
        for (int i = 0; i < 16; ++i)
            zo[64u * (16u * cq + i)] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
    }
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(tbase, kTcCols);
    }
}
