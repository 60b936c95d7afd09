// 16-qubit chunks on thread-block clusters, for states of 17..20 qubits
// (included inside qst.cu's anonymous namespace, after
// qst_tworound_packed.cuh, whose exchange layout and helpers it reuses).
//
// Binning settings by their high-bit pattern (Sec. III-B's per-setting
// rotations factor over qubits) shares the high factors of a bin's settings;
// above 16 qubits the 3^(n-12) patterns of a 12-qubit chunk outnumber the
// settings, so the chunk grows to 16 qubits (3^(n-16) <= 81 patterns, about 12
// settings per bin at n = 20, M = 1024).  A 2^16 chunk (512 KB) does not fit
// one SM: a work unit (bin, high pattern f, atom k) runs on a cluster of 8
// CTAs of 128 threads.  With the chunk index u = 4096 M + 64 H + L (M: chunk
// bits 12..15, H: 6..11, L: 0..5), CTA q holds rows M = 2q (threads 0..63)
// and 2q + 1 (threads 64..127), each as the two-round kernels hold a 12-qubit
// chunk:
//   round A: bits of H in registers (element i = H), thread t = L;
//   round B: bits of L in registers (element j = L), thread t = H (after the
//            exchange inside the 64 threads of the row);
//   round C: bits of M: thread tau of CTA q holds the 16 rows of the columns
//            H = 8 q + tau / 16, L = 4 (tau mod 16) + l, l < 4, as element
//            16 l + M, read from the row owners' exchange buffers through
//            distributed shared memory between two cluster barriers.
// The rotations' factors act on different qubits and commute, so the
// adjoint's inverse rounds run C, B, A, each with the same (Hermitian) factors.
//
// Round C's values sit in the CTA's own buffer at slot(M, H mod 8, L) =
// (M / 8) k2Buf + k2Row (8 (M mod 8) + H mod 8) + L: the same 8192 slots as
// the two-round exchange layout, so one 66 KB buffer serves every exchange
// (three CTAs per SM) and the cached adjoint's "all slots zero between
// settings" invariant covers both layouts.  An observed outcome u belongs to
// the CTA (u / 512) mod 8 that holds its column in round C: k_cl_partition
// groups each (setting, high pattern)'s observed entries by that CTA once per
// call, so a CTA walks only its own slice (and the transform cache is kept in
// that grouped order).
//
// Every CTA of a cluster runs the same unit, so the setting loops and the
// cluster barriers in them are uniform; a unit past the last bin leaves
// before the first barrier on all eight CTAs.

constexpr int kClChunk = 16;      // chunk bits of the cluster kernels
constexpr int kClCtas = 8;        // CTAs per cluster (two rows of 2^12 each)
constexpr uint32_t kClCols = 128; // TMEM columns of a CTA: the source (forward) or the accumulator (adjoint)

// The cluster CTAs take the two-round forward's shared memory and TMEM
// columns, so the occupancy and TMEM bounds proven for it cover them.
static_assert(kClCols == k2ColsFwd, "cluster CTAs are sized as two-round forward CTAs");

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Every thread of the cluster: this CTA's shared-memory writes are released,
// the other CTAs' acquired.
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Shared-memory address saddr of this CTA -> the same offset in CTA rank.
__device__ __forceinline__ uint32_t cl_map(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ float4 cl_ld4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

__host__ __device__ constexpr uint32_t cl_slot(uint32_t M, uint32_t Hl, uint32_t L) {
    return (M >> 3) * (uint32_t)k2Buf + (uint32_t)k2Row * (((M & 7u) << 3) | Hl) + L;
}
__host__ __device__ constexpr uint32_t cl_slot_u(uint32_t u) { return cl_slot(u >> 12, (u >> 6) & 7u, u & 63u); }
__host__ __device__ constexpr uint32_t cl_owner(uint32_t u) { return (u >> 9) & 7u; }
static_assert(cl_slot(15, 7, 63) + 1 == 2 * k2Buf - 2, "round C's slots are the exchange buffer's data slots");

constexpr int kClStage = 256;  // entries of a CTA's slice staged per setting (cp.async, double-buffered)
struct ClSmem {
    int work, stage_u, stage_p, masks, meta, tmem, total;
};
__host__ __device__ constexpr ClSmem cl_smem() {
    ClSmem sp{};
    sp.work = 0;
    sp.stage_u = sp.work + 2 * k2Buf * 8;          // [buffer][entry] chunk bits of the outcome
    sp.stage_p = sp.stage_u + 2 * kClStage * 4;    // [buffer][entry] CSR index
    sp.masks = sp.stage_p + 2 * kClStage * 4;
    sp.meta = sp.masks + kMaxBin * (int)sizeof(uint2);
    sp.tmem = sp.meta + kMaxBin * (int)sizeof(SetMeta);
    sp.total = sp.tmem + 16;
    return sp;
}
static_assert(cl_smem().stage_u % 16 == 0 && cl_smem().stage_p % 16 == 0 && cl_smem().masks % 16 == 0 &&
                  cl_smem().meta % 16 == 0,
              "aligned shared arrays");
// the same footprint as a two-round forward CTA: at most three per SM (384 TMEM columns)
static_assert(cl_smem().total == k2_smem_fwd().total, "cluster CTAs are sized as two-round forward CTAs");

// One warp per (setting s, high pattern f): the observed entries of chunk f
// (CSR range [a0, b0), outcomes ascending) grouped by owner CTA, stable:
// perm[a0 + i] = CSR index of the i-th entry in grouped order, pu[a0 + i] its
// outcome's chunk bits, ofs[(s 2^r + f) 9 + g] = where owner g's group starts
// (ofs[.. 8] = b0 - a0).
__global__ void __launch_bounds__(256) k_cl_partition(const int64_t *__restrict__ row_ptr,
                                                      const uint32_t *__restrict__ outcome,
                                                      const int32_t *__restrict__ choff, int M, int r,
                                                      int32_t *__restrict__ perm, uint32_t *__restrict__ pu,
                                                      int32_t *__restrict__ ofs) {
    __shared__ uint32_t next_sm[8][kClCtas];
    const int F = 1 << r;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u, wl = threadIdx.x >> 5;
    if (gw >= (int64_t)M * F) return;  // the whole warp
    const int s = (int)(gw / F), f = (int)(gw % F);
    const int64_t a0 = row_ptr[s] + choff[(size_t)s * (F + 1) + f];
    const int64_t b0 = row_ptr[s] + choff[(size_t)s * (F + 1) + f + 1];
    uint32_t tot = 0;  // lane g < 8: entries owned by CTA g
    for (int64_t j0 = a0; j0 < b0; j0 += 32) {
        const int64_t j = j0 + lane;
        const uint32_t g = j < b0 ? cl_owner(outcome[j]) : 8u;
#pragma unroll
        for (uint32_t h = 0; h < (uint32_t)kClCtas; ++h) {
            const uint32_t m = __ballot_sync(0xffffffffu, g == h);
            if (lane == h) tot += __popc(m);
        }
    }
    uint32_t incl = tot;  // inclusive prefix over lanes 0..7 (the other lanes hold 0)
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= (uint32_t)d) incl += o;
    }
    uint32_t *next = next_sm[wl];
    int32_t *og = ofs + (size_t)gw * (kClCtas + 1);
    if (lane < (uint32_t)kClCtas) {
        og[lane] = (int32_t)(incl - tot);
        next[lane] = incl - tot;
    }
    if (lane == kClCtas - 1) og[kClCtas] = (int32_t)incl;
    __syncwarp();
    for (int64_t j0 = a0; j0 < b0; j0 += 32) {
        const int64_t j = j0 + lane;
        const uint32_t u = j < b0 ? outcome[j] : 0u;
        const uint32_t g = j < b0 ? cl_owner(u) : 8u;
        const uint32_t peers = __match_any_sync(0xffffffffu, g);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        const uint32_t pos = g < 8u ? next[g] + rank : 0u;
        __syncwarp();
        if (g < 8u && rank == 0) next[g] += __popc(peers);
        __syncwarp();
        if (g < 8u) {
            perm[a0 + pos] = (int32_t)j;
            pu[a0 + pos] = u & ((1u << kClChunk) - 1u);
        }
    }
}

// The bin's masks and, per setting, this CTA's slice of chunk f's grouped
// entries (lo: first grouped index, cnt: its length) and 2^-m.
__device__ __forceinline__ void cl_stage_bin(const Bin &b, uint32_t f, int F, uint32_t q,
                                             const int32_t *__restrict__ order, const SetPlan *__restrict__ plans,
                                             const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ choff,
                                             const int32_t *__restrict__ ofs, uint2 *masks_sm, SetMeta *meta_sm) {
    for (int si = threadIdx.x; si < b.count; si += blockDim.x) {
        const int s = order[b.start + si];
        const SetPlan &P = plans[s];
        masks_sm[si] = make_uint2(P.xy, P.y);
        const int32_t *o = ofs + ((size_t)s * F + f) * (kClCtas + 1);
        SetMeta mt;
        mt.lo = (int32_t)(row_ptr[s] + choff[(size_t)s * (F + 1) + f] + o[q]);
        mt.cnt = o[q + 1] - o[q];
        mt.off = 0;
        mt.cs = exp2f(-(float)P.m);
        meta_sm[si] = mt;
    }
}

// Round C's four columns of every row, from the row owners (row M: CTA M / 2,
// buffer half M mod 2, row H, columns L0 .. L0 + 3).  off = byte offset of
// (H, L0) in a half buffer.
__device__ __forceinline__ void cl_load_C_remote(float2 (&v)[64], uint32_t wsa, uint32_t off) {
#pragma unroll
    for (int M = 0; M < 16; ++M) {
        const uint32_t ra = cl_map(wsa, (uint32_t)(M >> 1)) + (uint32_t)((M & 1) * k2Buf * 8) + off;
        const float4 x0 = cl_ld4(ra), x1 = cl_ld4(ra + 16u);
        v[M] = make_float2(x0.x, x0.y);
        v[16 + M] = make_float2(x0.z, x0.w);
        v[32 + M] = make_float2(x1.x, x1.y);
        v[48 + M] = make_float2(x1.z, x1.w);
    }
}
__device__ __forceinline__ void cl_store_C(const float2 (&v)[64], float2 *W, uint32_t Hl, uint32_t L0) {
#pragma unroll
    for (int M = 0; M < 16; ++M) {
        float4 *d = reinterpret_cast<float4 *>(W + cl_slot((uint32_t)M, Hl, L0));
        d[0] = make_float4(v[M].x, v[M].y, v[16 + M].x, v[16 + M].y);
        d[1] = make_float4(v[32 + M].x, v[32 + M].y, v[48 + M].x, v[48 + M].y);
    }
}
__device__ __forceinline__ void cl_load_C(float2 (&v)[64], const float2 *W, uint32_t Hl, uint32_t L0) {
#pragma unroll
    for (int M = 0; M < 16; ++M) {
        const float4 *s = reinterpret_cast<const float4 *>(W + cl_slot((uint32_t)M, Hl, L0));
        const float4 x0 = s[0], x1 = s[1];
        v[M] = make_float2(x0.x, x0.y);
        v[16 + M] = make_float2(x0.z, x0.w);
        v[32 + M] = make_float2(x1.x, x1.y);
        v[48 + M] = make_float2(x1.z, x1.w);
    }
}
// Row M, column block H of round B (64 consecutive slots) from the CTA that
// holds it in round C.
__device__ __forceinline__ void cl_load_B_remote(float2 (&v)[64], uint32_t wsa, uint32_t M, uint32_t H) {
    const uint32_t ra = cl_map(wsa, H >> 3) + 8u * cl_slot(M, H & 7u, 0u);
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
        const float4 x = cl_ld4(ra + 16u * jj);
        v[2 * jj] = make_float2(x.x, x.y);
        v[2 * jj + 1] = make_float2(x.z, x.w);
    }
}
// Round A's column of thread t, cleared behind the read.
__device__ __forceinline__ void cl_load_A_clear(float2 (&v)[64], float2 *wk, uint32_t t) {
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        v[i] = wk[k2Row * i + t];
        wk[k2Row * i + t] = make_float2(0.f, 0.f);
    }
}
// z += v for 128 TMEM columns (element i in columns 2i, 2i + 1), 32 at a time.
__device__ __forceinline__ void cl_tm_acc(uint32_t t_z, const float2 (&v)[64]) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        uint32_t r[32];
        tm_ld_issue(t_z + 32u * h, r);
        tm_ld_wait(r);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            r[2 * i] = __float_as_uint(__fadd_rn(__uint_as_float(r[2 * i]), v[16 * h + i].x));
            r[2 * i + 1] = __float_as_uint(__fadd_rn(__uint_as_float(r[2 * i + 1]), v[16 * h + i].y));
        }
        tm_st(t_z + 32u * h, r);
    }
    tm_wait_st();
}

// Unit of a cluster: consecutive clusters take consecutive atoms of one
// (bin, high pattern).
struct ClUnit {
    int k, bin;
    uint32_t f;
};
__device__ __forceinline__ ClUnit cl_unit(int K, int r) {
    const int unit = (int)(blockIdx.x / kClCtas);
    ClUnit u;
    u.k = unit % K;
    const int rest = unit / K;
    u.f = (uint32_t)rest & ((1u << r) - 1u);
    u.bin = rest >> r;
    return u;
}

// Forward.  Per setting: rounds A and B on the CTA's two rows, round B's rows
// published, round C's columns gathered, round C; the transforms (unscaled)
// then sit in the CTA's buffer at round C's slots, and the CTA gathers
// w_k 2^-m |.|^2 at its slice of the setting's observed outcomes (CACHE: also
// the transforms, into the atom's slice of a.phi_obs, in grouped order).
// Barriers per setting: one per row (the in-row exchange), two cluster
// barriers (round B published; every remote read done, so the buffer may be
// rewritten) and two block barriers (the staged slice and round C's values
// visible; the gather done before the next setting's exchange).
template <bool CACHE>
__global__ void __cluster_dims__(kClCtas, 1, 1) __launch_bounds__(k2T, 3) k_forward_cl(const FwdArgs a) {
    constexpr ClSmem sp = cl_smem();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *stage_u = reinterpret_cast<uint32_t *>(smem + sp.stage_u);
    int32_t *stage_p = reinterpret_cast<int32_t *>(smem + sp.stage_p);
    uint2 *masks_sm = reinterpret_cast<uint2 *>(smem + sp.masks);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    uint32_t *tmem_sm = reinterpret_cast<uint32_t *>(smem + sp.tmem);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, t = tid & 63u, half = tid >> 6;
    const uint32_t q = cl_rank();
    const ClUnit un = cl_unit(a.K, a.r);
    if (un.bin >= *a.n_bins || (a.skip && *a.skip)) return;  // the whole cluster
    const Bin b = a.bins[un.bin];
    const int D = 1 << a.n;
    const int k = un.k;
    const uint32_t f = un.f;
    const uint32_t Mrow = 2u * q + half;
    float2 *W = reinterpret_cast<float2 *>(smem + sp.work);
    float2 *wk = W + half * k2Buf;
    const uint32_t wsa = smem_u32(W);
    const uint32_t Hl = tid >> 4, L0 = 4u * (tid & 15u);
    const uint32_t offC = 8u * ((uint32_t)k2Row * (8u * q + Hl) + L0);
    if (warp == 0) tm_alloc(tmem_sm, kClCols);
    cl_stage_bin(b, f, 1 << a.r, q, a.order, a.plans, a.row_ptr, a.choff, a.cl_ofs, masks_sm, meta_sm);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t t_src = tmem_sm[0] + ((warp * 32u) << 16);
    const int bcount = b.count;
    const uint32_t *pu = a.cl_pu;
    const int32_t *perm = a.cl_perm;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            const int o = (si & 1) * kClStage;
            const int nst = mt.cnt < kClStage ? mt.cnt : kClStage;
            for (int j = tid; j < nst; j += k2T) {
                cp_async4(stage_u + o + j, pu + mt.lo + j);
                cp_async4(stage_p + o + j, perm + mt.lo + j);
            }
        }
        cp_async_commit();
    };
    const float wkk = a.w[k];
    float *pk = a.ppart + (size_t)k * a.nnz;
    issue(0);
    k2_build_source<12, kClChunk>(t_src, a.psi + (size_t)un.bin * a.src_bin_stride + (size_t)k * D + ((size_t)Mrow << 12),
                              true, f, b.xytop, b.ytop, t);
    tm_wait_st();
    for (int si = 0; si < bcount; ++si) {
        const uint2 mk = masks_sm[si];
        const SetMeta mt = meta_sm[si];
        float2 v[64];
        k2_tm_ld64(t_src, v);
        // rounds A, B, C share one butterfly site (code size)
#pragma unroll 1
        for (int R = 0; R < 3; ++R) {
            const uint32_t sh = R == 0 ? 6u : (R == 1 ? 0u : 12u), bits = R == 2 ? 15u : 63u;
            butterfly_herm<6>(v, (mk.x >> sh) & bits, (mk.y >> sh) & bits);
            if (R == 0) {
                k2_store_A(v, wk, t);
                k2_bar_atom(half);
                k2_load_B(v, wk, t);
            } else if (R == 1) {
                k2_store_B(v, wk, t);  // each thread rewrites the row only it read
                cl_sync();             // every row of the chunk is in round B
                cl_load_C_remote(v, wsa, offC);
                cl_sync();             // every remote read is done: buffers may be rewritten
            }
        }
        cl_store_C(v, W, Hl, L0);
        const float sc = wkk * mt.cs;
        cp_async_wait0();
        __syncthreads();  // this setting's stage landed (every thread's copies); round C's values are written
        // the stage buffer of setting si + 1 was last read by the gather of si - 1,
        // which every thread finished before the barrier above
        issue(si + 1);
        const uint32_t *su = stage_u + (si & 1) * kClStage;
        const int32_t *sq = stage_p + (si & 1) * kClStage;
        for (int j = tid; j < mt.cnt; j += k2T) {
            const bool st = j < kClStage;
            const uint32_t u = st ? su[j] : pu[mt.lo + j];
            const int32_t jj = st ? sq[j] : perm[mt.lo + j];
            const float2 ph = W[cl_slot_u(u)];
            pk[jj] = scaled_abs2(sc, ph);
            if (CACHE) a.phi_obs[(size_t)k * a.nnz + mt.lo + j] = ph;
        }
        if (a.p_dense) {  // every outcome of the CTA's columns
            const int s = a.order[b.start + si];
            float *pd = a.p_dense + (size_t)s * D + ((size_t)f << kClChunk);
            for (uint32_t e = tid; e < 8192u; e += k2T) {
                const uint32_t M = e >> 9, h = (e >> 6) & 7u, L = e & 63u;
                atomicAdd(pd + ((M << 12) | ((8u * q + h) << 6) | L), scaled_abs2(sc, W[cl_slot(M, h, L)]));
            }
        }
        __syncthreads();  // the gather is done before the next setting's exchange stores
    }
    cp_async_wait0();
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(tmem_sm[0], kClCols);
    }
}

// Adjoint from the transforms (the forward's phi at the observed outcomes, in
// a.phi_obs in grouped order): per setting, y = c 2^-m phi scattered into round
// C's slots (the buffer is all zero between settings), inverse round C, the
// columns written back and published, each row's round-B block gathered from
// its column's CTA, inverse round B, the exchange into round A (clearing every
// slot behind the reads), inverse round A, z += v in TMEM.  z is written once
// per unit, chunk f of the bin's slice of a.zbuf in round A's layout; k_reduce
// applies the bins' inverse high factors and sums them.
__global__ void __cluster_dims__(kClCtas, 1, 1) __launch_bounds__(k2T, 3) k_adjoint_clc(const AdjArgs a) {
    constexpr ClSmem sp = cl_smem();
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *stage_u = reinterpret_cast<uint32_t *>(smem + sp.stage_u);
    int32_t *stage_p = reinterpret_cast<int32_t *>(smem + sp.stage_p);
    uint2 *masks_sm = reinterpret_cast<uint2 *>(smem + sp.masks);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    uint32_t *tmem_sm = reinterpret_cast<uint32_t *>(smem + sp.tmem);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, t = tid & 63u, half = tid >> 6;
    const uint32_t q = cl_rank();
    const ClUnit un = cl_unit(a.K, a.r);
    if (un.bin >= *a.n_bins || (a.skip && *a.skip)) return;  // the whole cluster
    const Bin b = a.bins[un.bin];
    const int D = 1 << a.n;
    const int k = un.k;
    const uint32_t f = un.f;
    const uint32_t Mrow = 2u * q + half;
    float2 *W = reinterpret_cast<float2 *>(smem + sp.work);
    float2 *wk = W + half * k2Buf;
    const uint32_t wsa = smem_u32(W);
    const uint32_t Hl = tid >> 4, L0 = 4u * (tid & 15u);
    if (warp == 0) tm_alloc(tmem_sm, kClCols);
    for (int e = tid; e < 2 * k2Buf; e += k2T) W[e] = make_float2(0.f, 0.f);
    cl_stage_bin(b, f, 1 << a.r, q, a.order, a.plans, a.row_ptr, a.choff, a.cl_ofs, masks_sm, meta_sm);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t t_z = tmem_sm[0] + ((warp * 32u) << 16);
    {
        const uint32_t zero[32] = {};
#pragma unroll
        for (int h = 0; h < 4; ++h) tm_st(t_z + 32u * h, zero);
        tm_wait_st();
    }
    const int bcount = b.count;
    const uint32_t *pu = a.cl_pu;
    const int32_t *perm = a.cl_perm;
    const float *c_obs = a.c_obs;
    const float2 *phk = a.phi_obs + (size_t)k * a.nnz;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            const int o = (si & 1) * kClStage;
            const int nst = mt.cnt < kClStage ? mt.cnt : kClStage;
            for (int j = tid; j < nst; j += k2T) {
                cp_async4(stage_u + o + j, pu + mt.lo + j);
                cp_async4(stage_p + o + j, perm + mt.lo + j);
            }
        }
        cp_async_commit();
    };
    issue(0);
    float2 v[64];
    for (int si = 0; si < bcount; ++si) {
        const uint2 mk = masks_sm[si];
        const SetMeta mt = meta_sm[si];
        cp_async_wait0();
        __syncthreads();  // setting si's stage landed; setting si - 1's clears are done
        issue(si + 1);    // into the buffer last read by setting si - 1's scatter
        {
            const uint32_t *su = stage_u + (si & 1) * kClStage;
            const int32_t *sq = stage_p + (si & 1) * kClStage;
            for (int j = tid; j < mt.cnt; j += k2T) {
                const bool st = j < kClStage;
                const uint32_t u = st ? su[j] : pu[mt.lo + j];
                const int32_t jj = st ? sq[j] : perm[mt.lo + j];
                const float cy = c_obs[jj] * mt.cs;
                const float2 ph = phk[mt.lo + j];
                W[cl_slot_u(u)] = make_float2(cy * ph.x, cy * ph.y);
            }
        }
        __syncthreads();  // the scatter is visible
        cl_load_C(v, W, Hl, L0);
        // inverse rounds C, B, A (one butterfly site)
#pragma unroll 1
        for (int R = 0; R < 3; ++R) {
            const uint32_t sh = R == 0 ? 12u : (R == 1 ? 0u : 6u), bits = R == 0 ? 15u : 63u;
            butterfly_herm<6>(v, (mk.x >> sh) & bits, (mk.y >> sh) & bits);
            if (R == 0) {
                cl_store_C(v, W, Hl, L0);  // each thread rewrites the slots only it read
                cl_sync();                 // every column is in round C's output
                cl_load_B_remote(v, wsa, Mrow, t);
                cl_sync();                 // every remote read is done: buffers may be rewritten
            } else if (R == 1) {
                k2_store_B(v, wk, t);
                k2_bar_atom(half);
                cl_load_A_clear(v, wk, t);  // every slot of the row's half is cleared behind the reads
            }
        }
        cl_tm_acc(t_z, v);
    }
    cp_async_wait0();
    {
        float2 *zo = a.zbuf + ((size_t)un.bin * a.K + k) * D + ((size_t)f << kClChunk) + ((size_t)Mrow << 12) + t;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint32_t r[32];
            tm_ld_issue(t_z + 32u * h, r);
            tm_ld_wait(r);
#pragma unroll
            for (int i = 0; i < 16; ++i)
                zo[64u * (16 * h + i)] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
        }
    }
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(tmem_sm[0], kClCols);
    }
}
