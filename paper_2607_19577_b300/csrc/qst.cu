// qst.cu — sm_103a forward/adjoint of the local-Pauli measurement oracle of
// rank-adaptive matrix-free atomic quantum state tomography, behind the C ABI
// declared in include/qst.h.
//
// Method (paper Sec. II-III, Pauli POVM of Sec. IV):
//   forward  p_{s,u} = sum_k w_k |(V_s psi_k)_u|^2          (Eq. atomic-born-map)
//            c = pihat / (p/B + eps),  L = -sum pihat log(p/B + eps)
//                                                         (Eqs. qst-loss, likelihood-ratio-vector)
//   adjoint  G psi_k = (1/B) sum_s V_s^*(c_s .* V_s psi_k) (Eq. negative-gradient-product)
//            dJ/dpsi_k^* = -w_k G psi_k                    (Eq. atom-wirtinger-gradient)
//            dJ/dw_k = -h_k,  h_k = a(psi_k)^T c           (Eq. weight-gradient)
//
// Design (one GPU, matrix-free):
//   * V_s is a Kronecker product of 2x2 factors; Z factors are the identity and
//     X/Y factors are add-only butterflies once the 1/sqrt2 factors are pulled
//     out (the scale 2^-m_s, m_s = number of X/Y qubits, is applied once).
//   * The n outcome bits are split into c low "chunk" bits, transformed on-chip
//     (registers + shared memory), and r = n - c high bits.  Settings are binned
//     by their basis pattern on the high bits; every setting in a bin shares the
//     same high-bit factor U_h, so
//         sum_{s in bin} V_s^* y_s = (U_h^* (x) I) sum_{s in bin} (I (x) U_{L,s}^*) y_s.
//     A work unit (bin, high pattern f, atom k) therefore accumulates the inner
//     sum for its chunk in registers across all of the bin's settings, and a
//     reduction kernel applies U_h^* once per bin and sums the bins (compensated).
//     The high-bit factor of the forward is applied on load, once per unit.
//   * Inside a chunk each thread holds 2^A amplitudes (A = 5); a round applies
//     up to A X/Y qubits in registers, and rounds are joined by transposes
//     through XOR-swizzled shared memory.
//   * c is zero at unobserved outcomes; it is scattered into a dense chunk
//     buffer per setting and cleared again after use.
//   * No atomics on the data path: every sum has a fixed order.
#include "qst.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

namespace {

constexpr int kMaxChunk = 12;   // chunk bits transformed on-chip
constexpr int kMaxRounds = 3;   // 1 + ceil((kMaxChunk - A) / A) for A = 4, 5
constexpr int kDefaultRegBits = 4;  // 16 amplitudes per thread and round (measured faster than 32)
constexpr int kMaxTop = 4;      // high bits handled by binning (n <= 16)
constexpr int kMaxKeys = 81;    // 3^kMaxTop
constexpr int kMaxBin = 96;     // settings per bin (metadata staged in shared memory)
constexpr int kStage = 1024;    // observed entries per setting staged by cp.async

// Per-setting transform plan, written by k_pack.
struct SetPlan {
    uint32_t xy;               // outcome-bit mask of X/Y-measured qubits (all n bits)
    uint32_t y;                // outcome-bit mask of Y-measured qubits
    int32_t m;                 // popcount(xy)
    int32_t nr;                // rounds of the chunk transform
    uint32_t rdA[kMaxRounds];  // register bits of each round (see below)
    uint32_t rdB[kMaxRounds];  // thread bits of each round (see below)
    uint32_t key;              // base-3 basis pattern of the r high bits
    uint32_t pad;
    uint32_t p8[kMaxRounds][8];  // 8 * phys(1 << register position j) per round (j < A; 16-B rows)
};
// rdA: bits [4j, 4j+4) = chunk position of register bit j (j < 5), bits
// [20, 25) = register bits that are X/Y, bits [25, 30) = those that are Y.
// rdB: bits [4b, 4b+4) = chunk position of thread-index bit b (b < 7).  The
// four lowest thread bits are chosen with distinct positions mod 4, so the 16
// threads of a half-warp hit 16 distinct bank pairs under the swizzle below.

struct Bin {
    int32_t start;   // first index into the sorted setting order
    int32_t count;   // settings in the bin (<= kMaxBin)
    uint32_t xytop;  // high-bit X/Y mask, relative to bit c
    uint32_t ytop;   // high-bit Y mask, relative to bit c
};

// A bin setting's view of chunk f, staged in shared memory per work unit.
struct SetMeta {
    int32_t lo;      // first CSR index of the setting's outcomes in chunk f
    int32_t cnt;     // number of them
    int32_t off;     // prefix of cnt over the bin (forward p accumulator)
    float cs;        // 2^-m
};

// ----------------------------------------------------------------- device helpers

// Shared-memory XOR swizzle for complex64 arrays: the low 4 index bits are
// XOR-ed with bits 4..7 and 8..11.  It is GF(2)-linear, so the address of
// (base | offset) is phys(base) ^ phys(offset) for disjoint bit sets, and
// index bit b moves the bank pair by 2^(b mod 4).
__device__ __forceinline__ uint32_t phys(uint32_t u) {
    return u ^ (((u >> 4) ^ (u >> 8)) & 15u);
}

// Padded index of the fixed-round kernels (one spare element per 16): additive
// over disjoint bit sets, fx_pidx(a | b) = fx_pidx(a) + fx_pidx(b).
__host__ __device__ constexpr uint32_t fx_pidx(uint32_t u) { return u + (u >> 4); }

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Unscaled factors on register bit j, written in place (each output reuses
// its input's registers, so branches over the per-round bit pattern need no
// register copies at their merge points):
//   X:  (a, b) -> (a + b, a - b)            as  a += b;  b = a - 2b
//   Y:  (a, b) -> (a - i b, -i a + b)       as  a -= i b; b = 2b - i a
//   Y inverse: (a, b) -> (a + i b, i a + b) as  a += i b; b = 2b + i a
// The Y rows are those of V_Y = [[1,-i],[1,i]]/sqrt2 with the second row
// multiplied by -i.  That per-outcome phase leaves |(V_s psi)_u|^2 unchanged,
// and it cancels in V_s^* (c .* V_s psi) because diagonals commute, so both
// passes compute exactly the quantities of the paper.
template <int A>
__device__ __forceinline__ void butterfly_fwd(float2 (&v)[1 << A], uint32_t xyf, uint32_t yf) {
#pragma unroll
    for (int j = 0; j < A; ++j) {
        if (!((xyf >> j) & 1u)) continue;
        if ((yf >> j) & 1u) {
#pragma unroll
            for (int i = 0; i < (1 << A); ++i) {
                if ((i >> j) & 1) continue;
                float2 &a = v[i], &b = v[i | (1 << j)];
                a.x += b.y;
                a.y -= b.x;
                b.x = fmaf(2.f, b.x, a.y);
                b.y = fmaf(2.f, b.y, -a.x);
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

// Conjugate transposes of the factors above (X is its own).
template <int A>
__device__ __forceinline__ void butterfly_inv(float2 (&v)[1 << A], uint32_t xyf, uint32_t yf) {
#pragma unroll
    for (int j = 0; j < A; ++j) {
        if (!((xyf >> j) & 1u)) continue;
        if ((yf >> j) & 1u) {
#pragma unroll
            for (int i = 0; i < (1 << A); ++i) {
                if ((i >> j) & 1) continue;
                float2 &a = v[i], &b = v[i | (1 << j)];
                a.x -= b.y;
                a.y += b.x;
                b.x = fmaf(2.f, b.x, -a.y);
                b.y = fmaf(2.f, b.y, a.x);
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

// x * i^ph
__device__ __forceinline__ float2 mul_ipow(float2 x, int ph) {
    switch (ph & 3) {
        case 0: return x;
        case 1: return make_float2(-x.y, x.x);
        case 2: return make_float2(-x.x, -x.y);
        default: return make_float2(x.y, -x.x);
    }
}

// Scatter the low bits of src into the set bits of mask (software pdep).
__device__ __forceinline__ uint32_t pdep(uint32_t src, uint32_t mask) {
    uint32_t out = 0;
    for (uint32_t bb = 1; mask; bb <<= 1) {
        if (src & bb) out |= mask & (0u - mask);
        mask &= mask - 1;
    }
    return out;
}

// Block sum in a fixed order (deterministic), valid for any block size up to
// kRedMax, including blocks smaller than a warp.  Result valid in thread 0.
constexpr int kRedMax = 256;
template <typename Tv>
__device__ Tv block_sum(Tv x, Tv *scratch) {
    __syncthreads();
    scratch[threadIdx.x] = x;
    __syncthreads();
    Tv t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)blockDim.x; ++i) t += scratch[i];
    return t;
}

// Stage a bin's per-setting plans and chunk-f ranges in shared memory.
// Returns (in thread 0's view and, after the barrier, everyone's) the bin's
// total observed entries in chunk f.
__device__ __forceinline__ void stage_bin(const Bin &b, uint32_t f, int nf, const int32_t *__restrict__ order,
                                          const SetPlan *__restrict__ plans, const int64_t *__restrict__ row_ptr,
                                          const int32_t *__restrict__ choff, SetPlan *plans_sm, SetMeta *meta_sm,
                                          int *total_sm) {
    for (int si = threadIdx.x; si < b.count; si += blockDim.x) {
        const int s = order[b.start + si];
        const SetPlan P = plans[s];
        plans_sm[si] = P;
        const int64_t rb = row_ptr[s];
        const int32_t c0 = choff[(size_t)s * nf + f], c1 = choff[(size_t)s * nf + f + 1];
        SetMeta mt;
        mt.lo = (int32_t)(rb + c0);
        mt.cnt = c1 - c0;
        mt.off = 0;
        mt.cs = exp2f(-(float)P.m);
        meta_sm[si] = mt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int si = 0; si < b.count; ++si) {
            meta_sm[si].off = acc;
            acc += meta_sm[si].cnt;
        }
        *total_sm = acc;
    }
    __syncthreads();
}

// ----------------------------------------------------------------- kernels

// w 2^-m |z|^2 with every rounding fixed in the source (fma(re, re, im * im),
// then the scale), so kernels that share the expression give the same bits
// whatever contractions the compiler would choose in each.
__device__ __forceinline__ float scaled_abs2(float sc, float2 z) {
    return __fmul_rn(sc, __fmaf_rn(z.x, z.x, __fmul_rn(z.y, z.y)));
}

// Multi-instance launches (qst_batch): the CTAs of several instances' grids
// in one launch.  start[i] is the first CTA of instance i (ascending, start[0]
// = 0); a CTA finds its instance by binary search and runs the instance's
// kernel body with its CTA index within that instance's grid.
__device__ __forceinline__ int multi_find(const int *__restrict__ start, int count, int bid) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(start + mid) <= bid) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Descriptor packing (Sec. IV: Pauli strings) and setting binning: one block.
__device__ __forceinline__ void pack_body(const uint8_t *__restrict__ basis, int M, int n, int c, int r,
                                               int smax, int areg, SetPlan *__restrict__ plans,
                                               int32_t *__restrict__ order,
                                               Bin *__restrict__ bins, int *__restrict__ n_bins,
                                               int *__restrict__ status, const int cta) {
    __shared__ int hist[kMaxKeys], running[kMaxKeys];
    __shared__ int wcnt[32][kMaxKeys];
    const int tid = threadIdx.x;
    const int nkeys = (r == 0) ? 1 : (r == 1 ? 3 : (r == 2 ? 9 : (r == 3 ? 27 : 81)));
    const int A = c < areg ? c : areg;
    const int tb = c - A;  // thread-index bits
    for (int i = tid; i < kMaxKeys; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int s = tid; s < M; s += blockDim.x) {
        uint32_t xy = 0, y = 0, key = 0, p3 = 1;
        bool bad = false;
        for (int q = 0; q < n; ++q) {
            int code = basis[(size_t)s * n + q];
            if (code > 2) { bad = true; code = 0; }
            const int pos = n - 1 - q;
            if (code) xy |= 1u << pos;
            if (code == 2) y |= 1u << pos;
        }
        for (int j = 0; j < r; ++j) {
            const int pos = c + j;
            const int code = ((y >> pos) & 1u) ? 2 : (((xy >> pos) & 1u) ? 1 : 0);
            key += code * p3;
            p3 *= 3;
        }
        if (bad) atomicOr(status, QST_DEV_BAD_BASIS);
        SetPlan P;
        P.xy = xy;
        P.y = y;
        P.m = __popc(xy);
        P.key = key;
        P.pad = 0;
        // per-round plans of the generic kernels (chunks of <= 12 bits; the
        // cluster kernels' 16-bit chunks use the masks only)
        int nr = 0;
        if (c <= kMaxChunk) {
            // round 0: register bits = the top A chunk bits; thread bits ascending
            uint32_t wa = 0, wb = 0;
            for (int j = 0; j < A; ++j) wa |= (uint32_t)(c - A + j) << (4 * j);
            wa |= ((xy >> (c - A)) & ((1u << A) - 1u)) << 20;
            wa |= ((y >> (c - A)) & ((1u << A) - 1u)) << 25;
            for (int b = 0; b < tb; ++b) wb |= (uint32_t)b << (4 * b);
            P.rdA[0] = wa;
            P.rdB[0] = wb;
            nr = 1;
            uint32_t rem = xy & ((1u << (c - A)) - 1u);
            while (rem && nr < kMaxRounds) {
                uint32_t chosen = 0;
                int cnt = 0;
                while (rem && cnt < A) {
                    chosen |= rem & (0u - rem);
                    rem &= rem - 1;
                    ++cnt;
                }
                uint32_t regs = chosen;
                for (int pos = c - 1; __popc(regs) < A && pos >= 0; --pos) regs |= 1u << pos;  // identity pads
                uint32_t word = 0, xyf = 0, yf = 0;
                int j = 0;
                for (uint32_t cm = regs; cm; cm &= cm - 1, ++j) {
                    const int pos = __ffs(cm) - 1;
                    word |= (uint32_t)pos << (4 * j);
                    if ((chosen >> pos) & 1u) {
                        xyf |= 1u << j;
                        if ((y >> pos) & 1u) yf |= 1u << j;
                    }
                }
                // thread bits: lowest available position of each residue mod 4 first
                uint32_t avail = ((1u << c) - 1u) & ~regs, tw = 0;
                int b = 0;
                for (int res = 0; res < 4 && b < tb; ++res) {
                    for (int pos = res; pos < c; pos += 4) {
                        if ((avail >> pos) & 1u) {
                            tw |= (uint32_t)pos << (4 * b++);
                            avail &= ~(1u << pos);
                            break;
                        }
                    }
                }
                for (; avail && b < tb; avail &= avail - 1) tw |= (uint32_t)(__ffs(avail) - 1) << (4 * b++);
                P.rdA[nr] = word | (xyf << 20) | (yf << 25);
                P.rdB[nr] = tw;
                ++nr;
            }
        }
        for (int j = nr; j < kMaxRounds; ++j) P.rdA[j] = P.rdB[j] = 0;
        P.nr = nr;
        for (int j = 0; j < kMaxRounds; ++j)
            for (int q = 0; q < 8; ++q)
                P.p8[j][q] = (q < A && j < nr) ? phys(1u << ((P.rdA[j] >> (4 * q)) & 15u)) << 3 : 0u;
        plans[s] = P;
        atomicAdd(&hist[key], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int pos = 0, nb = 0;
        for (int key = 0; key < nkeys; ++key) {
            running[key] = pos;
            const int C = hist[key];
            uint32_t xyt = 0, yt = 0;
            int kk = key;
            for (int j = 0; j < r; ++j, kk /= 3) {
                const int d = kk % 3;
                if (d) xyt |= 1u << j;
                if (d == 2) yt |= 1u << j;
            }
            for (int j = 0; j < C; j += smax) {
                Bin b;
                b.start = pos + j;
                b.count = (C - j) < smax ? (C - j) : smax;
                b.xytop = xyt;
                b.ytop = yt;
                bins[nb++] = b;
            }
            pos += C;
        }
        *n_bins = nb;
    }
    __syncthreads();
    // Stable scatter of settings into key order.
    const int lane = tid & 31, wid = tid >> 5;
    for (int base = 0; base < M; base += blockDim.x) {
        const int s = base + tid;
        const uint32_t key = (s < M) ? plans[s].key : 0xffffffffu;
        for (int i = lane; i < nkeys; i += 32) wcnt[wid][i] = 0;
        __syncthreads();
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (s < M && lane == __ffs(peers) - 1) wcnt[wid][key] = __popc(peers);
        __syncthreads();
        for (int key2 = tid; key2 < nkeys; key2 += blockDim.x) {
            int acc = running[key2];
            for (int w = 0; w < 32; ++w) {
                const int t = wcnt[w][key2];
                wcnt[w][key2] = acc;
                acc += t;
            }
            running[key2] = acc;
        }
        __syncthreads();
        if (s < M) order[wcnt[wid][key] + rank] = s;
        __syncthreads();
    }
}
__global__ void __launch_bounds__(1024) k_pack(const uint8_t *__restrict__ basis, int M, int n, int c, int r,
                                               int smax, int areg, SetPlan *__restrict__ plans,
                                               int32_t *__restrict__ order,
                                               Bin *__restrict__ bins, int *__restrict__ n_bins,
                                               int *__restrict__ status) {
    pack_body(basis, M, n, c, r, smax, areg, plans, order, bins, n_bins, status, blockIdx.x);
}

// CSR validation and per-(setting, high pattern) offsets of the observed
// outcomes (outcomes are sorted, so each high pattern is a contiguous range).
// One warp per setting.  A malformed row is flagged and treated as empty.
__device__ __forceinline__ void validate_body(const int64_t *__restrict__ row_ptr, const uint32_t *__restrict__ outcome,
                           const uint32_t *__restrict__ shots, int M, int64_t nnz, int n, int c, int r,
                           int validate, int32_t *__restrict__ choff, int *__restrict__ status, const int cta) {
    const int gw = (cta * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= M) return;
    const int s = gw;
    const int nf = (1 << r) + 1;
    int32_t *co = choff + (size_t)s * nf;
    const int64_t lo = row_ptr[s], hi = row_ptr[s + 1];
    int bad = 0;
    if (validate) {
        if (lo < 0 || hi < lo || hi > nnz || (s == 0 && lo != 0) || (s == M - 1 && hi != nnz)) bad = QST_DEV_BAD_CSR;
        if (!bad && hi - lo > (1ll << n)) bad = QST_DEV_BAD_CSR;
        if (!bad) {
            const uint32_t D = 1u << n;
            for (int64_t j = lo + lane; j < hi; j += 32) {
                const uint32_t u = outcome[j];
                if (u >= D || (j > lo && u <= outcome[j - 1])) bad = QST_DEV_BAD_CSR;
            }
            if (shots && hi > lo && shots[s] == 0u) bad |= QST_DEV_BAD_SHOTS;
        }
        bad = __reduce_or_sync(0xffffffffu, bad);
    }
    if (bad) {
        if (lane == 0) atomicOr(status, bad);
        for (int f = lane; f < nf; f += 32) co[f] = 0;
        return;
    }
    for (int f = lane; f < nf; f += 32) {
        int64_t a = lo, b = hi;  // first j with (outcome[j] >> c) >= f
        while (a < b) {
            const int64_t mid = (a + b) >> 1;
            if ((int64_t)(outcome[mid] >> c) < f) a = mid + 1; else b = mid;
        }
        co[f] = (int32_t)(a - lo);
    }
}
__global__ void k_validate(const int64_t *__restrict__ row_ptr, const uint32_t *__restrict__ outcome,
                           const uint32_t *__restrict__ shots, int M, int64_t nnz, int n, int c, int r,
                           int validate, int32_t *__restrict__ choff, int *__restrict__ status) {
    validate_body(row_ptr, outcome, shots, M, nnz, n, c, r, validate, choff, status, blockIdx.x);
}

// Compile-time geometry of a chunk of 2^C amplitudes.
template <int C, int RA>
struct Geo {
    static constexpr int A = C < RA ? C : RA;        // register bits per round
    static constexpr int E = 1 << A;                 // amplitudes per thread
    static constexpr int TB = C - A;                 // thread-index bits
    static constexpr int T = 1 << TB;                // threads per unit
    static constexpr int N = 1 << C;                 // chunk size
};

__host__ __device__ constexpr int ctz_c(int t) { return (t & 1) ? 0 : 1 + ctz_c(t >> 1); }

// Gray-code walk over the 2^A register elements: within a chain, step t flips
// register bit ctz(t), so each element's offset is one XOR away from the
// previous one.  The low L register bits are walked by 2^(A-L) independent
// chains (one per value h of the high bits), which keeps the XOR dependency
// chains short.  Template recursion keeps every index a compile-time constant.
template <int L, int HI, int t>
struct GrayChain {
    template <int A, typename Fn>
    __device__ __forceinline__ static void run(uint32_t x, const uint32_t (&P8)[A], Fn &fn) {
        constexpr int j = ctz_c(t);
        x ^= P8[j];
        fn(std::integral_constant<int, (HI | (t ^ (t >> 1)))>(), x);
        GrayChain<L, HI, t + 1>::run(x, P8, fn);
    }
};
template <int L, int HI>
struct GrayChain<L, HI, (1 << L)> {
    template <int A, typename Fn>
    __device__ __forceinline__ static void run(uint32_t, const uint32_t (&)[A], Fn &) {}
};

template <int A, int L, int h>
struct GrayChains {
    template <typename Fn>
    __device__ __forceinline__ static void run(uint32_t b8, const uint32_t (&P8)[A], Fn &fn) {
        uint32_t x = b8;
#pragma unroll
        for (int j = 0; j < A - L; ++j)
            if ((h >> j) & 1) x ^= P8[L + j];
        fn(std::integral_constant<int, (h << L)>(), x);
        GrayChain<L, (h << L), 1>::run(x, P8, fn);
        GrayChains<A, L, h + 1>::run(b8, P8, fn);
    }
};
template <int A, int L>
struct GrayChains<A, L, (1 << (A - L))> {
    template <typename Fn>
    __device__ __forceinline__ static void run(uint32_t, const uint32_t (&)[A], Fn &) {}
};

// Thread -> amplitude mapping of one round, as byte offsets into a swizzled
// complex64 buffer: thread t holds the 2^A amplitudes whose register bits take
// every value and whose other chunk bits spell t.  Offsets are generated along
// a Gray code, one XOR per amplitude.
template <int C, int RA>
struct Lay {
    using G = Geo<C, RA>;
    uint32_t b8;          // 8 * phys(base of this thread)
    uint32_t P8[G::A];    // 8 * phys(1 << position of register bit j)
    uint32_t xyf, yf;     // which register bits are X/Y, Y
    // lut: this setting's per-round thread-offset tables (see build_lut)
    __device__ __forceinline__ void init(const SetPlan &P, int j, const uint32_t *lut, uint32_t tid) {
        const uint4 lo = *reinterpret_cast<const uint4 *>(&P.p8[j][0]);
        const uint4 hi = *reinterpret_cast<const uint4 *>(&P.p8[j][4]);
        const uint32_t all[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
        for (int q = 0; q < G::A; ++q) P8[q] = all[q];
        b8 = lut[j * 32 + (tid & 15u)] ^ lut[j * 32 + 16 + ((tid >> 4) & 15u)];
        const uint32_t rdA = P.rdA[j];
        xyf = (rdA >> 20) & 31u;
        yf = (rdA >> 25) & 31u;
    }
    // fn(integral_constant<i>, byte offset of register element i), every i once
    template <typename Fn>
    __device__ __forceinline__ void walk(Fn &&fn) const {
        constexpr int L = G::A < 3 ? G::A : 3;
        GrayChains<G::A, L, 0>::run(b8, P8, fn);
    }
};

__device__ __forceinline__ float2 lds2(const unsigned char *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void sts2(unsigned char *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

// Per-round thread-offset tables of one setting: for round j and each nibble
// value v, lut[32 j + v] = 8 phys(thread bits 0..3 = v) and
// lut[32 j + 16 + v] = 8 phys(thread bits 4..7 = v), placed at the round's
// thread-bit positions.  phys is GF(2)-linear, so a thread's base offset is
// the XOR of its two entries.
template <int TB>
__device__ __forceinline__ void build_lut(const SetPlan &P, uint32_t *lut, uint32_t tid, int T) {
    for (int e = tid; e < kMaxRounds * 32; e += T) {
        const int j = e >> 5, h = (e >> 4) & 1, nib = e & 15;
        const uint32_t rdB = P.rdB[j];
        uint32_t val = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int tb = 4 * h + b;
            if (((nib >> b) & 1) && tb < TB) val ^= phys(1u << ((rdB >> (4 * tb)) & 15u)) << 3;
        }
        lut[e] = val;
    }
}

// Chunk f of (U_h (x) I) psi_k in registers: element i of thread t is
// amplitude t + i 2^TB of the chunk.  U_h is the unscaled product of the
// high-bit factors, with the same rows as the butterflies (Z factors select
// f'_j = f_j).  Only elements I0 .. I0 + NI - 1 are built (a caller short of
// registers builds the chunk in parts).  CS: the chunk's own bits when the
// 2^C amplitudes built are one block of a larger chunk (psik then points at
// that block inside chunk 0).
template <int C, int RA, int I0 = 0, int NI = Geo<C, RA>::E, int CS = C>
__device__ __forceinline__ void build_source_regs(float2 (&acc)[Geo<C, RA>::E], const float2 *__restrict__ psik,
                                                  uint32_t f, uint32_t xytop, uint32_t ytop, uint32_t tid) {
    using G = Geo<C, RA>;
#pragma unroll
    for (int i = I0; i < I0 + NI; ++i) acc[i] = make_float2(0.f, 0.f);
    const int nx = __popc(xytop);
    // coefficient phase i^ph of source chunk f' in output chunk f
    auto chunk = [&](int idx, int &ph) {
        const uint32_t fp = (f & ~xytop) | pdep((uint32_t)idx, xytop);
        ph = 0;
        for (uint32_t mm = xytop; mm; mm &= mm - 1) {
            const int j = __ffs(mm) - 1;
            const uint32_t fj = (f >> j) & 1u, fpj = (fp >> j) & 1u;
            if ((ytop >> j) & 1u) {
                if (fj != fpj) ph += 3;  // Y rows [[1,-i],[-i,1]], as in the butterflies
            } else if (fj & fpj) {
                ph += 2;                 // X rows [[1,1],[1,-1]]
            }
        }
        return psik + ((size_t)fp << CS) + tid;
    };
    const int nidx = 1 << nx;
    int idx = 0;
    for (; idx + 1 < nidx; idx += 2) {  // two chunks in flight per step
        int ph0, ph1;
        const float2 *b0 = chunk(idx, ph0), *b1 = chunk(idx + 1, ph1);
        float2 x0[NI], x1[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            x0[i] = __ldg(b0 + ((I0 + i) << G::TB));
            x1[i] = __ldg(b1 + ((I0 + i) << G::TB));
        }
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const float2 y0 = mul_ipow(x0[i], ph0), y1 = mul_ipow(x1[i], ph1);
            acc[I0 + i].x += y0.x + y1.x;
            acc[I0 + i].y += y0.y + y1.y;
        }
    }
    if (idx < nidx) {
        int ph0;
        const float2 *b0 = chunk(idx, ph0);
#pragma unroll
        for (int i = I0; i < I0 + NI; ++i) {
            const float2 y0 = mul_ipow(__ldg(b0 + (i << G::TB)), ph0);
            acc[i].x += y0.x;
            acc[i].y += y0.y;
        }
    }
}

// The same chunk written to shared memory "i-major": register element i of
// thread t at index i 2^TB + t.
template <int C, int RA>
__device__ __forceinline__ void build_source(float2 *src, const float2 *__restrict__ psik, uint32_t f,
                                             uint32_t xytop, uint32_t ytop, uint32_t tid) {
    using G = Geo<C, RA>;
    float2 acc[G::E];
    build_source_regs<C, RA>(acc, psik, f, xytop, ytop, tid);
#pragma unroll
    for (int i = 0; i < G::E; ++i) src[(i << G::TB) + tid] = acc[i];
}

// Forward rounds of one setting's chunk transform.  On return v holds the
// transformed chunk in the layout of the last round, described by L.
template <int C, int RA>
__device__ __forceinline__ void forward_rounds(float2 (&v)[Geo<C, RA>::E], Lay<C, RA> &L, const SetPlan &P,
                                               const uint32_t *lut, const float2 *src, unsigned char *work,
                                               uint32_t tid) {
    using G = Geo<C, RA>;
    L.init(P, 0, lut, tid);
#pragma unroll
    for (int i = 0; i < G::E; ++i) v[i] = src[(i << G::TB) + tid];
    const int nr = P.nr;
    for (int j = 0;; ++j) {  // one butterfly site keeps the unrolled code small
        butterfly_fwd<G::A>(v, L.xyf, L.yf);
        if (j + 1 >= nr) break;
        __syncthreads();
        L.walk([&](auto ic, uint32_t x) { sts2(work + x, v[decltype(ic)::value]); });
        __syncthreads();
        L.init(P, j + 1, lut, tid);
        L.walk([&](auto ic, uint32_t x) { v[decltype(ic)::value] = lds2(work + x); });
    }
}

// Shared-memory plan of the two hot kernels (bytes, for a chunk of 2^c).
struct SmemPlan {
    int src, work, cden, stage, plans, meta, lut, total;
};
__host__ __device__ constexpr SmemPlan smem_plan(int c, bool adjoint) {
    SmemPlan sp{};
    sp.src = 0;
    sp.work = sp.src + (8 << c);
    sp.cden = sp.work + (8 << c);
    sp.stage = sp.cden + (adjoint ? (4 << c) : 0);
    sp.plans = sp.stage + 2 * kStage * (adjoint ? 8 : 4);
    sp.meta = sp.plans + kMaxBin * (int)sizeof(SetPlan);
    sp.lut = sp.meta + kMaxBin * (int)sizeof(SetMeta);
    sp.total = sp.lut + 2 * kMaxRounds * 32 * 4;
    return sp;
}

struct FwdArgs {
    const float2 *psi;
    const float *w;
    const SetPlan *plans;
    const int32_t *order;
    const Bin *bins;
    const int *n_bins;
    const int64_t *row_ptr;
    const uint32_t *outcome;
    const int32_t *choff;
    float *ppart;      // [K][nnz]: w_k |(V_s psi_k)_u|^2 at observed outcomes
    float *p_dense;    // optional [M][D] (accumulated with atomics; zeroed by the host)
    int64_t nnz;
    int64_t src_bin_stride;  // elements between the sources of consecutive bins (0: all bins read psi)
    const int *skip;         // optional device flag: when set, the launch does nothing
    int n, r, K;
    float2 *phi_obs = nullptr;  // optional [K][nnz]: the chunk transform of psi_k at the observed outcomes
    const unsigned char *tc_ops = nullptr;  // tensor-core kernels: the 729 group operators
    int *status = nullptr;                  // tensor-core kernels: QST_DEV_TIMEOUT
    // cluster kernels: each (setting, high pattern)'s observed entries grouped by the CTA
    // that holds their column (k_cl_partition)
    const int32_t *cl_perm = nullptr;
    const uint32_t *cl_pu = nullptr;
    const int32_t *cl_ofs = nullptr;
};

// Forward unit = (bin, high pattern f, atom k).  For every setting of the bin:
// the chunk of V_s psi_k, then w_k 2^-m |.|^2 at the setting's observed
// outcomes in chunk f, written to this atom's slice of the partial buffer.
// The next setting's outcome indices are prefetched with cp.async.
template <int C, int RA>
__device__ __forceinline__ void forward_body(const FwdArgs a, const int cta) {
    using G = Geo<C, RA>;
    constexpr SmemPlan sp = smem_plan(C, false);
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *src = reinterpret_cast<float2 *>(smem + sp.src);
    unsigned char *work = smem + sp.work;
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem + sp.stage);
    SetPlan *plans_sm = reinterpret_cast<SetPlan *>(smem + sp.plans);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    uint32_t *lut = reinterpret_cast<uint32_t *>(smem + sp.lut);
    __shared__ int total_sm;
    const uint32_t tid = threadIdx.x;
    const int unit = cta;
    const int k = unit % a.K;
    const int rest = unit / a.K;
    const uint32_t f = rest & ((1u << a.r) - 1u);
    const int bin = rest >> a.r;
    if (bin >= *a.n_bins || (a.skip && *a.skip)) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    constexpr uint32_t cmask = G::N - 1;
    constexpr int LUTW = kMaxRounds * 32;
    stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, plans_sm, meta_sm, &total_sm);
    const int bcount = b.count;
    const uint32_t *outcome = a.outcome;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            uint32_t *dst = stage + (si & 1) * kStage;
            const int nst = mt.cnt < kStage ? mt.cnt : kStage;
            for (int j = tid; j < nst; j += G::T) cp_async4(dst + j, outcome + mt.lo + j);
        }
        cp_async_commit();
    };
    const float wk = a.w[k];
    float *pk = a.ppart + (size_t)k * a.nnz;
    issue(0);
    build_source<C, RA>(src, a.psi + (size_t)bin * a.src_bin_stride + (size_t)k * D, f, b.xytop, b.ytop, tid);
    if (bcount > 0) build_lut<G::TB>(plans_sm[0], lut, tid, G::T);
    __syncthreads();
    for (int si = 0; si < bcount; ++si) {
        issue(si + 1);
        const SetPlan &P = plans_sm[si];
        const SetMeta mt = meta_sm[si];
        float2 v[G::E];
        Lay<C, RA> L;
        forward_rounds<C, RA>(v, L, P, lut + (si & 1) * LUTW, src, work, tid);
        cp_async_wait1();
        __syncthreads();
        L.walk([&](auto ic, uint32_t x) { sts2(work + x, v[decltype(ic)::value]); });
        __syncthreads();
        const float sc = wk * mt.cs;
        const uint32_t *st = stage + (si & 1) * kStage;
        for (int j = tid; j < mt.cnt; j += G::T) {
            const uint32_t u = (j < kStage ? st[j] : outcome[mt.lo + j]) & cmask;
            const float2 ph = lds2(work + (phys(u) << 3));
            pk[mt.lo + j] = scaled_abs2(sc, ph);
        }
        if (a.p_dense) {
            const int s = a.order[b.start + si];
            float *pd = a.p_dense + (size_t)s * D + ((size_t)f << C);
            for (uint32_t u = tid; u <= cmask; u += G::T) {
                const float2 ph = lds2(work + (phys(u) << 3));
                atomicAdd(pd + u, scaled_abs2(sc, ph));
            }
        }
        if (si + 1 < bcount) build_lut<G::TB>(plans_sm[si + 1], lut + ((si + 1) & 1) * LUTW, tid, G::T);
        __syncthreads();  // stage buffer and work are reused by the next setting
    }
    cp_async_wait0();
}
template <int C, int RA>
__global__ void __launch_bounds__(Geo<C, RA>::T, 2) k_forward(const FwdArgs a) {
    forward_body<C, RA>(a, blockIdx.x);
}
template <int C, int RA>
__global__ void __launch_bounds__(Geo<C, RA>::T, 2) k_forward_multi(const FwdArgs *__restrict__ args, const int *__restrict__ start, int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const FwdArgs a = args[i];
    forward_body<C, RA>(a, (int)blockIdx.x - start[i]);
}

// Forward epilogue, one warp per setting: p = sum_k of the atom partials
// (fixed order), pi = p / B, c = pihat / (pi + eps) and the loss terms
// -pihat log(pi + eps) (Eqs. qst-loss, likelihood-ratio-vector).  Per-block
// FP64 loss partials are summed by k_loss.  UNROLL (the batch's launch over
// all instances' settings): four atoms' loads in flight, added in the same
// order; on the n = 16 workload's single launch the plain loop measured faster
// (0.166 against 0.225 ms), on the 64-instance batch the unrolled one (15.48
// against 15.85 ms per evaluation).
template <bool UNROLL = false>
__device__ __forceinline__ void epilogue_body(const float *__restrict__ ppart, const int64_t *__restrict__ row_ptr,
                                                      const uint32_t *__restrict__ count,
                                                      const uint32_t *__restrict__ shots,
                                                      int M, int K, int64_t nnz, float invB, float eps,
                                                      float *__restrict__ p_obs, float *__restrict__ c_obs,
                                                      double *__restrict__ loss_part, const int *skip, const int cta) {
    if (skip && *skip) return;
    __shared__ double red[kRedMax];
    const int s = (cta * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    double lsum = 0.0;
    if (s < M) {
        const int64_t lo = row_ptr[s], hi = row_ptr[s + 1];
        // rows flagged malformed by the validation are skipped (their offsets were emptied)
        const bool ok = lo >= 0 && hi >= lo && hi <= nnz && shots[s] > 0u;
        if (ok) {
            const float ns = (float)shots[s];
            for (int64_t i = lo + lane; i < hi; i += 32) {
                float p = 0.f;
                if (UNROLL) {
                    const float *pp = ppart + i;
#pragma unroll 4
                    for (int k = 0; k < K; ++k, pp += nnz) p = __fadd_rn(p, *pp);
                } else {
                    for (int k = 0; k < K; ++k) p += ppart[(size_t)k * nnz + i];
                }
                const float den = __fadd_rn(__fmul_rn(p, invB), eps);  // pi + eps
                const float pihat = __fdiv_rn(__fmul_rn((float)count[i], invB), ns);
                if (c_obs) c_obs[i] = __fdiv_rn(pihat, den);
                if (p_obs) p_obs[i] = p;
                lsum = fma(-(double)pihat, (double)logf(den), lsum);
            }
        }
    }
    const double t = block_sum<double>(lsum, red);
    if (threadIdx.x == 0) loss_part[cta] = t;
}
__global__ void __launch_bounds__(256) k_fwd_epilogue(const float *__restrict__ ppart, const int64_t *__restrict__ row_ptr,
                                                      const uint32_t *__restrict__ count,
                                                      const uint32_t *__restrict__ shots,
                                                      int M, int K, int64_t nnz, float invB, float eps,
                                                      float *__restrict__ p_obs, float *__restrict__ c_obs,
                                                      double *__restrict__ loss_part, const int *skip) {
    epilogue_body(ppart, row_ptr, count, shots, M, K, nnz, invB, eps, p_obs, c_obs, loss_part, skip, blockIdx.x);
}

// d_k = -grad_k + w_k grad_w_k psi_k = w_k (I - psi_k psi_k^*) G psi_k
// (Eq. atom-projected-descent-direction), one thread per amplitude.
__global__ void __launch_bounds__(256) k_tangent(const float2 *__restrict__ psi, const float *__restrict__ w,
                                                 const float2 *grad, const float *__restrict__ gw, float2 *d,
                                                 int n, int K) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ((int64_t)K << n)) return;
    const int k = (int)(idx >> n);
    const float s = w[k] * gw[k];
    const float2 g = grad[idx], x = psi[idx];
    d[idx] = make_float2(fmaf(s, x.x, -g.x), fmaf(s, x.y, -g.y));
}

struct AdjArgs {
    const float2 *psi;
    const SetPlan *plans;
    const int32_t *order;
    const Bin *bins;
    const int *n_bins;
    const int64_t *row_ptr;
    const uint32_t *outcome;
    const float *c_obs;
    const int32_t *choff;
    float2 *zbuf;    // [bins][K][D]
    int64_t src_bin_stride;  // elements between the sources of consecutive bins (0: all bins read psi)
    int n, r, K;
    const float2 *phi_obs = nullptr;  // [K][nnz] from the forward (the cached adjoint reads it instead of psi)
    int64_t nnz = 0;
    const int *skip = nullptr;        // optional device flag: when set, the launch does nothing
    const unsigned char *tc_ops = nullptr;  // tensor-core kernels: the 729 group operators
    int *status = nullptr;                  // tensor-core kernels: QST_DEV_TIMEOUT
    const int32_t *cl_perm = nullptr;       // cluster kernels, as in FwdArgs
    const uint32_t *cl_pu = nullptr;
    const int32_t *cl_ofs = nullptr;
};

// Adjoint unit = (bin, high pattern f, atom k).  For every setting of the bin:
// recompute the chunk of V_s psi_k, multiply by c_s 2^-m (h partial sums on
// the way), apply the conjugate-transposed chunk rounds in reverse, and add
// into the register-resident accumulator z (round-0 layout).  The next
// setting's (outcome, c) pairs are prefetched with cp.async and scattered into
// the dense c buffer at the end of the current setting.
template <int C, int RA>
__device__ __forceinline__ void adjoint_body(const AdjArgs a, const int cta) {
    if (a.skip && *a.skip) return;
    using G = Geo<C, RA>;
    constexpr SmemPlan sp = smem_plan(C, true);
    extern __shared__ __align__(16) unsigned char smem[];
    const float2 *src = reinterpret_cast<const float2 *>(smem + sp.src);
    unsigned char *work = smem + sp.work;
    unsigned char *cdb = smem + sp.cden;  // float per amplitude, swizzled index
    uint32_t *stage_u = reinterpret_cast<uint32_t *>(smem + sp.stage);
    float *stage_c = reinterpret_cast<float *>(smem + sp.stage + 2 * kStage * 4);
    SetPlan *plans_sm = reinterpret_cast<SetPlan *>(smem + sp.plans);
    SetMeta *meta_sm = reinterpret_cast<SetMeta *>(smem + sp.meta);
    uint32_t *lut = reinterpret_cast<uint32_t *>(smem + sp.lut);
    __shared__ int total_sm;
    const uint32_t tid = threadIdx.x;
    const int unit = cta;
    const int k = unit % a.K;
    const int rest = unit / a.K;
    const uint32_t f = rest & ((1u << a.r) - 1u);
    const int bin = rest >> a.r;
    if (bin >= *a.n_bins) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    constexpr uint32_t cmask = G::N - 1;
    constexpr int LUTW = kMaxRounds * 32;
    float *cden = reinterpret_cast<float *>(cdb);
    for (uint32_t u = tid; u <= cmask; u += G::T) cden[u] = 0.f;
    stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, plans_sm, meta_sm, &total_sm);
    const int bcount = b.count;
    const uint32_t *outcome = a.outcome;
    const float *c_obs = a.c_obs;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            const int nst = mt.cnt < kStage ? mt.cnt : kStage;
            uint32_t *du = stage_u + (si & 1) * kStage;
            float *dc = stage_c + (si & 1) * kStage;
            for (int j = tid; j < nst; j += G::T) {
                cp_async4(du + j, outcome + mt.lo + j);
                cp_async4(dc + j, c_obs + mt.lo + j);
            }
        }
        cp_async_commit();
    };
    // scatter (val = c 2^-m) or clear (val = 0) setting si's entries of the
    // dense c buffer; each thread touches the entries it staged itself.
    auto scatter = [=](int si, bool clear) {
        const SetMeta mt = meta_sm[si];
        const uint32_t *su = stage_u + (si & 1) * kStage;
        const float *sc = stage_c + (si & 1) * kStage;
        for (int j = tid; j < mt.cnt; j += G::T) {
            const bool st = j < kStage;
            const uint32_t u = (st ? su[j] : outcome[mt.lo + j]) & cmask;
            cden[phys(u)] = clear ? 0.f : (st ? sc[j] : c_obs[mt.lo + j]) * mt.cs;
        }
    };
    issue(0);
    build_source<C, RA>(const_cast<float2 *>(src), a.psi + (size_t)bin * a.src_bin_stride + (size_t)k * D, f, b.xytop,
                        b.ytop, tid);
    if (bcount > 0) build_lut<G::TB>(plans_sm[0], lut, tid, G::T);
    cp_async_wait0();
    __syncthreads();  // c buffer zeroed, source built, round tables ready
    if (bcount > 0) scatter(0, false);
    float2 z[G::E];
#pragma unroll
    for (int i = 0; i < G::E; ++i) z[i] = make_float2(0.f, 0.f);
    for (int si = 0; si < b.count; ++si) {
        issue(si + 1);
        const SetPlan &P = plans_sm[si];
        const int nr = P.nr;
        const uint32_t *lt = lut + (si & 1) * LUTW;
        float2 v[G::E];
        Lay<C, RA> L;
        forward_rounds<C, RA>(v, L, P, lt, src, work, tid);
        if (nr == 1) __syncthreads();  // this setting's c scatter is visible
        L.walk([&](auto ic, uint32_t x) {
            constexpr int i = decltype(ic)::value;
            const float cc = *reinterpret_cast<const float *>(cdb + (x >> 1));
            v[i].x = __fmul_rn(v[i].x, cc);  // not contracted into the butterflies that follow
            v[i].y = __fmul_rn(v[i].y, cc);
        });
        for (int j = nr - 1;; --j) {  // one butterfly site
            butterfly_inv<G::A>(v, L.xyf, L.yf);
            if (j == 0) break;
            __syncthreads();
            L.walk([&](auto ic, uint32_t x) { sts2(work + x, v[decltype(ic)::value]); });
            __syncthreads();
            L.init(P, j - 1, lt, tid);
            L.walk([&](auto ic, uint32_t x) { v[decltype(ic)::value] = lds2(work + x); });
        }
#pragma unroll
        for (int i = 0; i < G::E; ++i) {
            z[i].x += v[i].x;
            z[i].y += v[i].y;
        }
        if (nr == 1) __syncthreads();  // every thread is done reading the c buffer
        scatter(si, true);
        if (si + 1 < bcount) build_lut<G::TB>(plans_sm[si + 1], lut + ((si + 1) & 1) * LUTW, tid, G::T);
        cp_async_wait0();
        __syncthreads();  // cleared before the next scatter; stage free for reuse; next tables ready
        if (si + 1 < b.count) scatter(si + 1, false);
    }
    float2 *zo = a.zbuf + ((size_t)bin * a.K + k) * D + ((size_t)f << C);
#pragma unroll
    for (int i = 0; i < G::E; ++i) zo[tid + (i << G::TB)] = z[i];
}
template <int C, int RA>
__global__ void __launch_bounds__(Geo<C, RA>::T, 2) k_adjoint(const AdjArgs a) {
    adjoint_body<C, RA>(a, blockIdx.x);
}
template <int C, int RA>
__global__ void __launch_bounds__(Geo<C, RA>::T, 2) k_adjoint_multi(const AdjArgs *__restrict__ args, const int *__restrict__ start, int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const AdjArgs a = args[i];
    adjoint_body<C, RA>(a, (int)blockIdx.x - start[i]);
}

// grad_k[f, l] = -(w_k / B) sum_bins (U_h^* z_{bin,k})[f, l]: the high-bit
// conjugate-transposed factors per bin, Kahan-compensated sum over bins.
template <int R>
__device__ __forceinline__ void reduce_body(const float2 *__restrict__ zbuf, const Bin *__restrict__ bins,
                                                const int *__restrict__ n_bins, const float *__restrict__ w,
                                                const float2 *__restrict__ psi, float2 *__restrict__ grad,
                                                double *__restrict__ hdot, int n, int c, int K, float invB,
                                                const int *skip, const int cta) {
    if (skip && *skip) return;
    constexpr int F = 1 << R;
    const int64_t idx = (int64_t)cta * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)K << c;
    if (idx >= total) return;
    const int k = (int)(idx >> c);
    const uint32_t ul = (uint32_t)(idx & ((1 << c) - 1));
    const int D = 1 << n;
    float2 acc[F], cmp[F];
#pragma unroll
    for (int f = 0; f < F; ++f) acc[f] = cmp[f] = make_float2(0.f, 0.f);
    const int nb = *n_bins;
    for (int bi = 0; bi < nb; ++bi) {
        const Bin b = bins[bi];
        const float2 *zp = zbuf + ((size_t)bi * K + k) * D + ul;
        float2 v[F];
#pragma unroll
        for (int f = 0; f < F; ++f) v[f] = zp[(size_t)f << c];
        butterfly_inv<R>(v, b.xytop, b.ytop);
#pragma unroll
        for (int f = 0; f < F; ++f) {
            float yv = v[f].x - cmp[f].x, tv = acc[f].x + yv;
            cmp[f].x = (tv - acc[f].x) - yv;
            acc[f].x = tv;
            yv = v[f].y - cmp[f].y;
            tv = acc[f].y + yv;
            cmp[f].y = (tv - acc[f].y) - yv;
            acc[f].y = tv;
        }
    }
    const float sc = -w[k] * invB;
    float2 *gp = grad + (size_t)k * D + ul;
    const float2 *pp = psi + (size_t)k * D + ul;
    double hd = 0.0;  // Re <psi_k | B G psi_k> over this thread's amplitudes
#pragma unroll
    for (int f = 0; f < F; ++f) {
        gp[(size_t)f << c] = make_float2(sc * acc[f].x, sc * acc[f].y);
        const float2 q = pp[(size_t)f << c];
        hd = fma((double)q.y, (double)acc[f].y, fma((double)q.x, (double)acc[f].x, hd));
    }
    hdot[idx] = hd;
}
template <int R>
__global__ void __launch_bounds__(256) k_reduce(const float2 *__restrict__ zbuf, const Bin *__restrict__ bins,
                                                const int *__restrict__ n_bins, const float *__restrict__ w,
                                                const float2 *__restrict__ psi, float2 *__restrict__ grad,
                                                double *__restrict__ hdot, int n, int c, int K, float invB,
                                                const int *skip) {
    reduce_body<R>(zbuf, bins, n_bins, w, psi, grad, hdot, n, c, K, invB, skip, blockIdx.x);
}

// grad_w_k = -h_k with h_k = a(psi_k)^T c = <psi_k | G psi_k> (Eqs. weight-gradient,
// atom-response): the FP64 sum of the reduction kernel's per-thread partials.
__device__ __forceinline__ void hsum_body(const double *__restrict__ hdot, int c, float invB,
                                              float *__restrict__ grad_w, const int *skip, const int cta) {
    if (skip && *skip) return;
    __shared__ double red[kRedMax];
    const int k = cta;
    const double *hp = hdot + ((size_t)k << c);
    double s = 0.0;
    for (int u = threadIdx.x; u < (1 << c); u += blockDim.x) s += hp[u];
    const double t = block_sum<double>(s, red);
    if (threadIdx.x == 0) grad_w[k] = (float)(-t * (double)invB);
}
__global__ void __launch_bounds__(256) k_hsum(const double *__restrict__ hdot, int c, float invB,
                                              float *__restrict__ grad_w, const int *skip) {
    hsum_body(hdot, c, invB, grad_w, skip, blockIdx.x);
}

// loss = sum of the forward epilogue's per-block partial sums (FP64, fixed order).
__device__ __forceinline__ void loss_body(const double *__restrict__ loss_part, int parts,
                                              double *__restrict__ loss, int *__restrict__ status, const int *skip, const int cta) {
    if (skip && *skip) return;
    __shared__ double red[kRedMax];
    double s = 0.0;
    for (int u = threadIdx.x; u < parts; u += blockDim.x) s += loss_part[u];
    const double t = block_sum<double>(s, red);
    if (threadIdx.x == 0) {
        if (loss) *loss = t;
        if (!isfinite(t)) atomicOr(status, QST_DEV_NONFINITE);
    }
}
__global__ void __launch_bounds__(256) k_loss(const double *__restrict__ loss_part, int parts,
                                              double *__restrict__ loss, int *__restrict__ status, const int *skip) {
    loss_body(loss_part, parts, loss, status, skip, blockIdx.x);
}

#include "qst_update.cuh"
#include "qst_spectral.cuh"
#include "qst_wide.cuh"
#include "qst_fixed.cuh"
#include "qst_tworound.cuh"
#include "qst_tworound_packed.cuh"
#include "qst_cluster.cuh"
#include "qst_warp.cuh"
#include "qst_tensorcore.cuh"
#include "qst_single.cuh"
#include "qst_iterate.cuh"

// ----------------------------------------------------------------- host side

int ipow3(int r) {
    int v = 1;
    for (int i = 0; i < r; ++i) v *= 3;
    return v;
}

}  // namespace

struct TimedLaunch {
    int kind;
    cudaEvent_t start, stop;
};

struct qst_plan_s {
    int n = 0, M = 0, K = 0, c = 0, r = 0, A = 0, T = 0, smax = 0, nb_max = 0, B = 0;
    bool wide = false;       // n = 17..20: high bits by butterfly passes, groups of wide_G settings
    bool fx = false;         // 12-qubit chunks with fixed-position rounds (k_forward_fx / k_adjoint_fx)
    bool fx2 = false;        // 12-qubit chunks in two 6-bit rounds, two atoms per CTA (k_forward_2r / k_adjoint_2r)
    int sms = 148;           // SMs of the plan's device (persistent grids)
    bool fw = false;         // states of 5..9 qubits in one chunk: a warp per (bin, atom) (k_forward_wu / k_adjoint_wu)
    bool cl = false;         // n = 17..20: 16-qubit chunks on 8-CTA clusters (k_forward_cl / k_adjoint_clc)
    int32_t *cl_perm = nullptr;   // [nnz] cluster kernels: CSR index of each entry in owner-grouped order
    uint32_t *cl_pu = nullptr;    // [nnz] its outcome's chunk bits
    int32_t *cl_ofs = nullptr;    // [M][2^r][kClCtas + 1] group starts within each (setting, high pattern)
    float2 *phi = nullptr;   // [K][nnz] transform cache of qst_evaluate (two-round plans, params.phi_cache)
    bool cache_on = false;   // qst_evaluate passes phi from the forward to the adjoint
    unsigned char *tc_ops = nullptr;  // precision > 0: the 729 six-qubit group operators (B operand layout)
    int wide_G = 0;
    float2 *wide_T = nullptr;    // [wide_G][K][D] intermediate (also the z buffer)
    double2 *wide_acc = nullptr; // [K][D] FP64 accumulator of G psi
    int64_t nnz = 0;
    qst_params prm{};
    int device = 0;
    // workspace
    SetPlan *plans = nullptr;
    int32_t *order = nullptr;
    Bin *bins = nullptr;
    int *n_bins = nullptr;
    int32_t *choff = nullptr;
    float *ppart = nullptr;
    double *loss_part = nullptr;
    int loss_parts = 0;
    float2 *zbuf = nullptr;
    double *hdot = nullptr;
    double2 *refac_C = nullptr;  // K x K Gram (refactorisation)
    double2 *refac_T = nullptr;  // K x K combination matrix
    // qst_step workspace
    float2 *step_trial = nullptr;  // [K][D] trial atoms
    float2 *step_grad = nullptr;   // [K][D] G psi
    float *step_c = nullptr;       // [nnz] likelihood ratio of the current state
    float *step_gw = nullptr;      // [K] weight gradient
    float *step_tw = nullptr;      // [K] trial weights
    float *step_m1 = nullptr;      // [K] all -1 (adjoint weights that return G psi)
    double *step_loss = nullptr;   // [1]
    int *step_kout = nullptr;      // [1]
    int *status = nullptr;
    // spectral step (block Krylov): basis, S times basis, work block, small matrices
    float2 *lz_Q = nullptr, *lz_SQ = nullptr, *lz_W = nullptr;
    double2 *lz_C = nullptr, *lz_P = nullptr, *lz_G = nullptr, *lz_Tm = nullptr, *lz_T = nullptr, *lz_Y = nullptr,
            *lz_Tc = nullptr;
    double *lz_lam = nullptr;
    int *lz_int = nullptr;  // [0] kept count, [1] selected s
    int lz_blocks = 0;            // Krylov blocks (adjoint launches) of the last spectral candidate
    double *it_Jseg = nullptr;    // qst_iterate with spectral slots: a graph segment's J / acceptance history
    int *it_aseg = nullptr;
    int it_seg_cap = 0;
    long long step_calls = 0;     // serial-equivalent oracle calls of the last qst_step slot 3
    // qst_iterate: device state, trial likelihood ratio, captured graph
    IterState *it_state = nullptr;
    float *it_c = nullptr;
    cudaStream_t it_cap = nullptr, it_body = nullptr;  // capture streams (main graph, conditional bodies)
    cudaGraphExec_t it_exec = nullptr;
    std::vector<double> it_key;
    int64_t it_launches = 0;
    int64_t ws_bytes = 0;
    // host-buffer path (allocated on first use)
    void *h_dev = nullptr;
    cudaStream_t h_side = nullptr;  // qst_evaluate_host: the counts' copy beside the forward
    cudaEvent_t h_fork = nullptr, h_count = nullptr;
    // accounting
    bool timing = false;
    std::vector<TimedLaunch> pending;
    std::vector<cudaEvent_t> pool;
    int64_t launches[QST_KERNEL_KINDS] = {0};
    double ms[QST_KERNEL_KINDS] = {0};
    int64_t total_launches = 0;
};

namespace {

template <typename Tp>
qst_status dalloc(qst_plan p, Tp **ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc((void **)ptr, count * sizeof(Tp)) != cudaSuccess) {
        cudaGetLastError();
        return QST_ERR_NO_MEMORY;
    }
    p->ws_bytes += (int64_t)(count * sizeof(Tp));
    return QST_OK;
}

cudaEvent_t take_event(qst_plan p) {
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

template <typename Fn>
qst_status launch(qst_plan p, int kind, cudaStream_t st, Fn &&fn) {
    TimedLaunch tl{kind, nullptr, nullptr};
    if (p->timing) {
        tl.start = take_event(p);
        tl.stop = take_event(p);
        cudaEventRecord(tl.start, st);
    }
    fn();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "qst: kernel launch failed: %s\n", cudaGetErrorString(e));
        return QST_ERR_CUDA;
    }
    if (p->timing) {
        cudaEventRecord(tl.stop, st);
        p->pending.push_back(tl);
    }
    p->total_launches++;
    return QST_OK;
}

void resolve_pending(qst_plan p) {
    for (auto &tl : p->pending) {
        cudaEventSynchronize(tl.stop);
        float t = 0.f;
        cudaEventElapsedTime(&t, tl.start, tl.stop);
        p->launches[tl.kind]++;
        p->ms[tl.kind] += t;
        p->pool.push_back(tl.start);
        p->pool.push_back(tl.stop);
    }
    p->pending.clear();
}

bool aligned(const void *ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

template <int C, int RA>
void set_smem_attrs() {
    cudaFuncSetAttribute(k_forward<C, RA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem_plan(C, false).total);
    cudaFuncSetAttribute(k_adjoint<C, RA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem_plan(C, true).total);
}

template <int C, typename Fn>
void with_ra(int ra, Fn &&fn) {
    if (ra == 4 || C <= 4) fn(std::integral_constant<int, C>(), std::integral_constant<int, 4>());
    else fn(std::integral_constant<int, C>(), std::integral_constant<int, 5>());
}

// Calls fn(integral_constant<C>, integral_constant<RA>) for the plan's chunk
// size and register bits (RA = 4 or 5; chunks below 5 bits use A = C).
template <typename Fn>
void with_geo(int c, int ra, Fn &&fn) {
    switch (c) {
        case 1: with_ra<1>(ra, fn); break;
        case 2: with_ra<2>(ra, fn); break;
        case 3: with_ra<3>(ra, fn); break;
        case 4: with_ra<4>(ra, fn); break;
        case 5: with_ra<5>(ra, fn); break;
        case 6: with_ra<6>(ra, fn); break;
        case 7: with_ra<7>(ra, fn); break;
        case 8: with_ra<8>(ra, fn); break;
        case 9: with_ra<9>(ra, fn); break;
        case 10: with_ra<10>(ra, fn); break;
        case 11: with_ra<11>(ra, fn); break;
        default: with_ra<12>(ra, fn); break;
    }
}

// The plan's forward / adjoint chunk kernel over `units` work units per atom
// (bins x high patterns): one CTA per unit and atom, or per unit and atom
// pair for the two-round kernels.
// Tensor-core kernels of a two-round plan with precision T = 1..3.
template <int T>
void launch_forward_tc(const FwdArgs &a, int grid, cudaStream_t st) {
    if (a.phi_obs) k_forward_tc<T, true><<<grid, kTcT, kTcSmemAlloc, st>>>(a);
    else k_forward_tc<T, false><<<grid, kTcT, kTcSmemAlloc, st>>>(a);
}
void launch_forward_units(qst_plan p, const FwdArgs &a0, int units, cudaStream_t st) {
    FwdArgs a = a0;
    a.tc_ops = p->tc_ops;
    a.status = p->status;
    a.cl_perm = p->cl_perm;
    a.cl_pu = p->cl_pu;
    a.cl_ofs = p->cl_ofs;
    if (p->fx2 && p->prm.precision > 0) {
        const int grid = units * ((p->K + 1) / 2);
        if (p->prm.precision == 1) launch_forward_tc<1>(a, grid, st);
        else if (p->prm.precision == 2) launch_forward_tc<2>(a, grid, st);
        else launch_forward_tc<3>(a, grid, st);
        return;
    }
    if (p->fw) {
        const int grid = (int)(((int64_t)units * p->K + kWuT / 32 - 1) / (kWuT / 32));
        with_wu(p->n, [&](auto nb) {
            constexpr int NB = decltype(nb)::value;
            k_forward_wu<NB><<<grid, kWuT, wu_smem(NB), st>>>(a);
        });
        return;
    }
    if (p->cl) {
        const int grid = units * p->K * kClCtas;
        if (a.phi_obs) k_forward_cl<true><<<grid, k2T, cl_smem().total, st>>>(a);
        else k_forward_cl<false><<<grid, k2T, cl_smem().total, st>>>(a);
        return;
    }
    if (p->fx2) {
        const int grid = units * k2_atom_groups(p->K, p->c);
        with_chunk2(p->c, [&](auto cc) {
            constexpr int C = decltype(cc)::value;
            if (a.phi_obs) k_forward_2r<true, C><<<grid, k2T, k2_smem_fwd().total, st>>>(a);
            else k_forward_2r<false, C><<<grid, k2T, k2_smem_fwd().total, st>>>(a);
        });
        return;
    }
    const int grid = units * p->K;
    if (p->fx && p->wide) {  // single-setting units, persistent CTAs (three per SM)
        const int pg = grid < 3 * p->sms ? grid : 3 * p->sms;
        if (a.phi_obs) k_forward_fx1p<true><<<pg, kFxT, kFx1pFwdSmem, st>>>(a);
        else k_forward_fx1p<false><<<pg, kFxT, kFx1pFwdSmem, st>>>(a);
        return;
    }
    if (p->fx) {
        k_forward_fx<<<grid, kFxT, fx_smem(false).total, st>>>(a);
        return;
    }
    with_geo(p->c, p->A, [&](auto cc, auto ra) {
        constexpr int C = decltype(cc)::value, RA = decltype(ra)::value;
        k_forward<C, RA><<<grid, Geo<C, RA>::T, smem_plan(C, false).total, st>>>(a);
    });
}
void launch_adjoint_units(qst_plan p, const AdjArgs &a0, int units, cudaStream_t st) {
    AdjArgs a = a0;
    a.tc_ops = p->tc_ops;
    a.status = p->status;
    a.cl_perm = p->cl_perm;
    a.cl_pu = p->cl_pu;
    a.cl_ofs = p->cl_ofs;
    if (p->fx2 && p->prm.precision > 0) {  // adjoint_core supplies the transforms
        const int grid = units * ((p->K + 1) / 2);
        if (p->prm.precision == 1) k_adjoint_tc<1><<<grid, kTcT, kTcSmemAlloc, st>>>(a);
        else if (p->prm.precision == 2) k_adjoint_tc<2><<<grid, kTcT, kTcSmemAlloc, st>>>(a);
        else k_adjoint_tc<3><<<grid, kTcT, kTcSmemAlloc, st>>>(a);
        return;
    }
    if (p->fw) {
        const int grid = (int)(((int64_t)units * p->K + kWuT / 32 - 1) / (kWuT / 32));
        with_wu(p->n, [&](auto nb) {
            constexpr int NB = decltype(nb)::value;
            k_adjoint_wu<NB><<<grid, kWuT, wu_smem(NB), st>>>(a);
        });
        return;
    }
    if (p->cl) {  // adjoint_core supplies the transforms
        k_adjoint_clc<<<units * p->K * kClCtas, k2T, cl_smem().total, st>>>(a);
        return;
    }
    if (p->fx2 && a.phi_obs) {
        const int grid = units * k2_atom_groups(p->K, p->c);
        with_chunk2(p->c, [&](auto cc) {
            constexpr int C = decltype(cc)::value;
            k_adjoint_2c<C><<<grid, k2T, k2c_smem(k2cStageSingle).total, st>>>(a);
        });
        return;
    }
    if (p->fx2) {
        const int grid = units * k2_atom_groups(p->K, p->c);
        with_chunk2(p->c, [&](auto cc) {
            constexpr int C = decltype(cc)::value;
            k_adjoint_2r<C><<<grid, k2T, k2p_smem().total, st>>>(a);
        });
        return;
    }
    const int grid = units * p->K;
    if (p->fx && p->wide) {  // single-setting units, persistent CTAs (four / two per SM)
        if (a.phi_obs) {
            const int pg = grid < 4 * p->sms ? grid : 4 * p->sms;
            k_adjoint_fx1cp<<<pg, kFxT, kFx1pAdjcSmem, st>>>(a);
        } else {
            const int pg = grid < 2 * p->sms ? grid : 2 * p->sms;
            k_adjoint_fx1p<<<pg, kFxT, kFx1pAdjSmem, st>>>(a);
        }
        return;
    }
    if (p->fx) {
        k_adjoint_fx<<<grid, kFxT, fx_smem(true).total, st>>>(a);
        return;
    }
    with_geo(p->c, p->A, [&](auto cc, auto ra) {
        constexpr int C = decltype(cc)::value, RA = decltype(ra)::value;
        k_adjoint<C, RA><<<grid, Geo<C, RA>::T, smem_plan(C, true).total, st>>>(a);
    });
}

qst_status prepare(qst_plan p, const uint8_t *basis, const int64_t *row_ptr, const uint32_t *outcome,
                   const uint32_t *shots, cudaStream_t st) {
    qst_status rc = launch(p, QST_KERNEL_PACK, st, [&] {
        // the wide path does not bin by the high pattern: one key, one bin
        k_pack<<<1, 1024, 0, st>>>(basis, p->M, p->n, p->c, p->wide ? 0 : p->r, p->wide ? p->M : p->smax, p->A,
                                   p->plans, p->order, p->bins, p->n_bins, p->status);
    });
    if (rc) return rc;
    const int warps_per_block = 8;
    const int grid = (p->M + warps_per_block - 1) / warps_per_block;
    rc = launch(p, QST_KERNEL_VALIDATE, st, [&] {
        k_validate<<<grid, 32 * warps_per_block, 0, st>>>(row_ptr, outcome, shots, p->M, p->nnz, p->n, p->c,
                                                          p->r, p->prm.validate, p->choff, p->status);
    });
    if (rc || !p->cl) return rc;
    const int64_t pairs = (int64_t)p->M << p->r;
    return launch(p, QST_KERNEL_VALIDATE, st, [&] {
        k_cl_partition<<<(int)((pairs + 7) / 8), 256, 0, st>>>(row_ptr, outcome, p->choff, p->M, p->r, p->cl_perm,
                                                               p->cl_pu, p->cl_ofs);
    });
}

}  // namespace

namespace {

// Wide path, forward: per atom and group of settings, the high pass into the
// intermediate, then the chunk kernel on single-setting bins reading it.
qst_status forward_wide(qst_plan p, const float2 *psi, const float *w, const int64_t *row_ptr,
                        const uint32_t *outcome, float *p_dense, cudaStream_t st, float2 *phi_cache) {
    const size_t D = (size_t)1 << p->n;
    const int tiles = (1 << p->c) / kWideCols;
    for (int g0 = 0; g0 < p->M; g0 += p->wide_G) {
        const int G = (p->M - g0) < p->wide_G ? (p->M - g0) : p->wide_G;
        qst_status rc = launch(p, QST_KERNEL_HIGH, st, [&] {
            k_high_fwd<<<dim3(tiles, p->K), kWideT, kWideSmem, st>>>(psi, p->plans, g0, G, p->K, p->c, p->wide_T);
        });
        if (!rc) rc = launch(p, QST_KERNEL_HIGH, st, [&] { k_wide_bins<<<1, 256, 0, st>>>(g0, G, p->bins, p->n_bins); });
        if (rc) return rc;
        FwdArgs a;
        a.psi = p->wide_T;
        a.w = w;
        a.plans = p->plans;
        a.order = p->order;
        a.bins = p->bins;
        a.n_bins = p->n_bins;
        a.row_ptr = row_ptr;
        a.outcome = outcome;
        a.choff = p->choff;
        a.ppart = p->ppart;
        a.p_dense = p_dense;
        a.nnz = p->nnz;
        a.src_bin_stride = (int64_t)p->K * (int64_t)D;
        a.skip = nullptr;
        a.n = p->n;
        a.r = p->r;
        a.K = p->K;
        a.phi_obs = phi_cache;
        const int units = G << p->r;
        rc = launch(p, QST_KERNEL_FORWARD, st, [&] {
            launch_forward_units(p, a, units, st);
        });
        if (rc) return rc;
    }
    return QST_OK;
}

// Wide path, adjoint: per atom and group, high pass, chunk adjoint writing z
// in place over the intermediate, inverse high pass accumulating into the FP64
// accumulator; then grad = -(w/B) acc and the h partials.
qst_status adjoint_wide(qst_plan p, const float2 *psi, const float *w, const int64_t *row_ptr,
                        const uint32_t *outcome, const float *c_obs, float2 *grad, cudaStream_t st,
                        const float2 *phi_cache) {
    const size_t D = (size_t)1 << p->n;
    const int tiles = (1 << p->c) / kWideCols;
    if (cudaMemsetAsync(p->wide_acc, 0, sizeof(double2) * (size_t)p->K * D, st) != cudaSuccess) return QST_ERR_CUDA;
    for (int g0 = 0; g0 < p->M; g0 += p->wide_G) {
        const int G = (p->M - g0) < p->wide_G ? (p->M - g0) : p->wide_G;
        qst_status rc = QST_OK;
        if (!phi_cache)  // with the transform cache the chunk adjoint needs no source
            rc = launch(p, QST_KERNEL_HIGH, st, [&] {
                k_high_fwd<<<dim3(tiles, p->K), kWideT, kWideSmem, st>>>(psi, p->plans, g0, G, p->K, p->c, p->wide_T);
            });
        if (!rc) rc = launch(p, QST_KERNEL_HIGH, st, [&] { k_wide_bins<<<1, 256, 0, st>>>(g0, G, p->bins, p->n_bins); });
        if (rc) return rc;
        AdjArgs a;
        a.psi = p->wide_T;
        a.plans = p->plans;
        a.order = p->order;
        a.bins = p->bins;
        a.n_bins = p->n_bins;
        a.row_ptr = row_ptr;
        a.outcome = outcome;
        a.c_obs = c_obs;
        a.choff = p->choff;
        a.zbuf = p->wide_T;  // each unit reads its chunk before writing its z over it
        a.src_bin_stride = (int64_t)p->K * (int64_t)D;
        a.n = p->n;
        a.r = p->r;
        a.K = p->K;
        a.phi_obs = phi_cache;
        a.nnz = p->nnz;
        const int units = G << p->r;
        rc = launch(p, QST_KERNEL_ADJOINT, st, [&] {
            launch_adjoint_units(p, a, units, st);
        });
        if (!rc) rc = launch(p, QST_KERNEL_HIGH, st, [&] {
            k_high_inv_acc<<<dim3(tiles, p->K), kWideT, kWideInvSmem, st>>>(p->wide_T, p->plans, g0, G, p->K, p->c,
                                                                          p->wide_acc);
        });
        if (rc) return rc;
    }
    const float invB = 1.0f / (float)p->B;
    const int64_t total = (int64_t)p->K << p->c;
    return launch(p, QST_KERNEL_REDUCE, st, [&] {
        k_wide_final<<<(int)((total + 255) / 256), 256, 0, st>>>(p->wide_acc, w, psi, grad, p->hdot, p->n, p->c,
                                                                 p->K, invB);
    });
}

qst_status forward_core(qst_plan p, const float *psi, const float *w, const int64_t *row_ptr, const uint32_t *outcome,
                        const uint32_t *count, const uint32_t *shots, float *p_obs, float *c_obs, double *loss,
                        float *p_dense, const int *skip, cudaStream_t st, float2 *phi_cache = nullptr,
                        cudaEvent_t count_ready = nullptr);
qst_status adjoint_core(qst_plan p, const float *psi, const float *w, const int64_t *row_ptr, const uint32_t *outcome,
                        const float *c_obs, float *grad_psi, float *grad_w, cudaStream_t st,
                        const float2 *phi_cache = nullptr, const int *skip = nullptr);
}  // namespace

extern "C" {

void qst_params_default(qst_params *p) {
    if (!p) return;
    p->eps = 1e-8;
    p->norm_settings = 0;
    p->chunk_qubits = 0;
    p->max_bin_settings = 0;
    p->validate = 1;
    p->reg_bits = 0;
    p->fixed_rounds = -1;
    p->phi_cache = -1;
    p->precision = 0;
}

const char *qst_status_string(qst_status s) {
    switch (s) {
        case QST_OK: return "ok";
        case QST_ERR_INVALID_ARG: return "invalid argument";
        case QST_ERR_UNSUPPORTED: return "unsupported size";
        case QST_ERR_CUDA: return "CUDA error";
        case QST_ERR_NO_MEMORY: return "out of device memory";
        case QST_ERR_DEVICE: return "device-side error";
        case QST_ERR_SCRATCH_TOO_SMALL: return "problem exceeds the no-allocation scratch";
    }
    return "unknown status";
}

qst_status qst_plan_create(qst_plan *out, int n, int M, int K, int64_t nnz, const qst_params *params) {
    if (!out) return QST_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || M < 1 || K < 1 || nnz < 0) return QST_ERR_INVALID_ARG;
    if (nnz > (int64_t)M << n) return QST_ERR_INVALID_ARG;
    qst_params prm;
    qst_params_default(&prm);
    if (params) prm = *params;
    if (!(prm.eps >= 0.0) || prm.norm_settings < 0 || prm.max_bin_settings < 0) return QST_ERR_INVALID_ARG;
    if (n > 16 + 4) return QST_ERR_UNSUPPORTED;
    // n <= 16: chunk min(n, 12), up to 4 binned high bits; n = 17..20: the wide
    // path (chunk n - 8, the 8 high bits applied by butterfly passes) or, asked
    // for with chunk_qubits = 16, 16-qubit chunks on thread-block clusters with
    // n - 16 binned high bits (measured slower: 154.8 against 76.8 ms per
    // evaluation of n = 20, M = 1024, K = 8).
    const int c_default = n <= 16 ? (n < kMaxChunk ? n : kMaxChunk) : n - kWideR;
    int c = prm.chunk_qubits ? prm.chunk_qubits : (n > 16 && prm.fixed_rounds == 4 ? kClChunk : c_default);
    const bool cl = n > 16 && c == kClChunk;
    if (!cl && (c < 1 || c > kMaxChunk || c > n)) return QST_ERR_INVALID_ARG;
    const int r = n - c;
    const bool wide = !cl && r > kMaxTop;
    if (wide && (r != kWideR || c < 9)) return QST_ERR_UNSUPPORTED;
    if (K > 4096 || M > (1 << 24) || nnz > ((int64_t)1 << 31) - 1) return QST_ERR_UNSUPPORTED;
    qst_plan p = new (std::nothrow) qst_plan_s;
    if (!p) return QST_ERR_NO_MEMORY;
    p->n = n;
    p->M = M;
    p->K = K;
    p->nnz = nnz;
    p->prm = prm;
    p->c = c;
    p->r = r;
    p->cl = cl;
    const int ra = prm.reg_bits ? prm.reg_bits : kDefaultRegBits;
    if (ra != 4 && ra != 5) {
        delete p;
        return QST_ERR_INVALID_ARG;
    }
    p->A = c < ra ? c : ra;
    p->T = 1 << (c - p->A);
    if (prm.fixed_rounds < -1 || prm.fixed_rounds > 4 || prm.phi_cache < -1 || prm.phi_cache > 1 ||
        prm.precision < 0 || prm.precision > 3) {
        delete p;
        return QST_ERR_INVALID_ARG;
    }
    p->B = prm.norm_settings ? prm.norm_settings : M;
    cudaGetDevice(&p->device);
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    p->sms = sms;
    if (prm.max_bin_settings) {
        p->smax = prm.max_bin_settings;
    } else {
        const int64_t target = (int64_t)sms * 16;
        int64_t s = ((int64_t)M * ((int64_t)1 << r) * K + target - 1) / target;
        p->smax = (int)(s < 4 ? 4 : s);
    }
    if (p->smax > kMaxBin) p->smax = kMaxBin;
    // 12-qubit chunk kernels.  The two-round kernels build a 64-amplitude-per-
    // thread source per unit at 8-12 warps per SM; that pays off only when a
    // unit runs many settings.  Automatic choice (-1): two rounds when bins may
    // hold >= 32 settings, else three (n = 12 instances with ~8 settings per
    // bin measured ~20 % faster with three rounds).  The wide path's units hold
    // one setting each: it always runs the three-round kernels (264 against
    // 356 ms on the n = 20 workload).
    // Whole states of 10, 11 qubits run the two-round kernels; their transform
    // cache (8 bytes per observed entry and atom) pays only when at most a quarter
    // of the outcomes are observed, so qst_evaluate's adjoint reads it there and
    // recomputes otherwise (phi_cache -1).
    const bool sparse = (int64_t)nnz * 4 <= ((int64_t)M << c);
    const int fr = prm.fixed_rounds >= 0 ? prm.fixed_rounds : (c < 12 && r == 0 && c >= 10 ? 2 : (p->smax >= 32 ? 2 : 1));
    // the cluster kernels are the 16-qubit chunks' only kernels (fixed_rounds 4, or automatic)
    if (cl != (prm.fixed_rounds == 4 || (cl && prm.fixed_rounds == -1))) {
        delete p;
        return QST_ERR_UNSUPPORTED;
    }
    // two-round kernels: 12-qubit chunks, and whole states of 10, 11 qubits (chunks of 10, 11)
    p->fx2 = (c == 12 || (c >= 10 && c < 12 && r == 0)) && fr == 2 && !wide && !cl;
    p->fx = c == 12 && p->A == 4 && (fr == 1 || (fr == 2 && wide));
    // whole states of 5..9 qubits: warp-per-unit kernels unless per-setting rounds are asked for
    // (0); from 10 qubits on a lane's 32 amplitudes and accumulator need ~250 registers and the
    // CTA kernels measured faster (3.3 against 1.8 ms on the batched workload's n = 10 instances)
    p->fw = !wide && r == 0 && c >= 5 && c <= kWuMaxQubits && (prm.fixed_rounds == -1 || prm.fixed_rounds == 3);
    if (prm.fixed_rounds == 3 && !p->fw) {
        delete p;
        return QST_ERR_UNSUPPORTED;
    }
    // the cached adjoint exists for the two-round kernels and the wide path's single-setting
    // 12-qubit-chunk kernels (n = 20)
    if (prm.phi_cache == 1 && !p->fx2 && !(wide && p->fx) && !cl) {
        delete p;
        return QST_ERR_UNSUPPORTED;
    }
    // the tensor-core chunk transforms exist for the two-round plans of 12-qubit chunks
    if (prm.precision > 0 && !(p->fx2 && c == 12)) {
        delete p;
        return QST_ERR_UNSUPPORTED;
    }
    const int64_t D = (int64_t)1 << n;
    if (wide) {
        p->wide = true;
        const int64_t g = kWideGroupBytes / (D * (int64_t)K * (int64_t)sizeof(float2));
        p->wide_G = (int)(g < 1 ? 1 : (g > M ? M : g));
        p->nb_max = p->wide_G;
    } else {
        const int nkeys = ipow3(r);
        p->nb_max = (nkeys < M ? nkeys : M) + (M + p->smax - 1) / p->smax;
    }
    p->loss_parts = (M + 7) / 8;  // forward epilogue: one warp per setting, 8 warps per block
    qst_status rc = QST_OK;
    if (!rc) rc = dalloc(p, &p->plans, M);
    if (!rc) rc = dalloc(p, &p->order, M);
    if (!rc) rc = dalloc(p, &p->bins, p->nb_max);
    if (!rc) rc = dalloc(p, &p->n_bins, 1);
    if (!rc) rc = dalloc(p, &p->choff, (size_t)M * ((1 << r) + 1));
    if (!rc) rc = dalloc(p, &p->ppart, (size_t)K * nnz);
    if (!rc) rc = dalloc(p, &p->loss_part, p->loss_parts);
    if (!rc && !wide) rc = dalloc(p, &p->zbuf, (size_t)p->nb_max * K * D);
    if (!rc && wide) rc = dalloc(p, &p->wide_T, (size_t)p->wide_G * K * D);
    if (!rc && wide) rc = dalloc(p, &p->wide_acc, (size_t)K * D);
    if (!rc && wide) p->zbuf = p->wide_T;
    if (!rc) rc = dalloc(p, &p->hdot, (size_t)K << c);
    if (!rc && cl) rc = dalloc(p, &p->cl_perm, nnz);
    if (!rc && cl) rc = dalloc(p, &p->cl_pu, nnz);
    if (!rc && cl) rc = dalloc(p, &p->cl_ofs, (size_t)M * ((size_t)1 << r) * (kClCtas + 1));
    if (!rc && K <= kRefacMax) rc = dalloc(p, &p->refac_C, (size_t)K * K);
    if (!rc && K <= kRefacMax) rc = dalloc(p, &p->refac_T, (size_t)K * K);
    if (!rc) rc = dalloc(p, &p->step_trial, (size_t)K * D);
    if (!rc) rc = dalloc(p, &p->step_grad, (size_t)K * D);
    if (!rc) rc = dalloc(p, &p->step_c, nnz);
    if (!rc) rc = dalloc(p, &p->step_gw, K);
    if (!rc) rc = dalloc(p, &p->step_tw, K);
    if (!rc) rc = dalloc(p, &p->step_m1, K);
    if (!rc) rc = dalloc(p, &p->step_loss, 1);
    if (!rc) rc = dalloc(p, &p->step_kout, 1);
    if (!rc && !wide && !cl && K <= kRefacMax / 2) {  // the spectral step needs >= 2 Krylov blocks
        const size_t nv = (size_t)(kKrylovMax + K);
        rc = dalloc(p, &p->lz_Q, nv * D);
        if (!rc) rc = dalloc(p, &p->lz_SQ, nv * D);
        if (!rc) rc = dalloc(p, &p->lz_W, (size_t)K * D);
        if (!rc) rc = dalloc(p, &p->lz_C, nv * kKrylovMax);
        if (!rc) rc = dalloc(p, &p->lz_P, (size_t)K * K);
        if (!rc) rc = dalloc(p, &p->lz_G, (size_t)K * K);
        if (!rc) rc = dalloc(p, &p->lz_Tm, (size_t)K * K);
        if (!rc) rc = dalloc(p, &p->lz_T, (size_t)kKrylovMax * kKrylovMax);
        if (!rc) rc = dalloc(p, &p->lz_Y, (size_t)kKrylovMax * kKrylovMax);
        if (!rc) rc = dalloc(p, &p->lz_Tc, (size_t)kKrylovMax * K);
        if (!rc) rc = dalloc(p, &p->lz_lam, kKrylovMax);
        if (!rc) rc = dalloc(p, &p->lz_int, 2);
    }
    // qst_evaluate's transform cache: K x nnz complex values (1 GB for the
    // n = 16, M = 4096, K = 16 workload); automatic for two-round plans up to 16 GiB
    // (for whole states of 10, 11 qubits only with sparse outcomes; on the wide path
    // with 12-qubit chunks, n = 20, only when asked for: there the adjoint recomputes
    // by default); always held by cluster plans, whose adjoint reads transforms
    if (!rc && nnz > 0 &&
        ((p->fx2 && (prm.phi_cache == 1 || (prm.phi_cache == -1 && (int64_t)K * nnz * 8 <= ((int64_t)16 << 30) &&
                                            (c == 12 || sparse)))) ||
         (wide && p->fx && prm.phi_cache == 1) || (p->fx2 && prm.precision > 0) || cl))
        rc = dalloc(p, &p->phi, (size_t)K * nnz);
    // with precision > 0 the buffer is also the tensor-core adjoint's input when the cache is off
    // (the cluster kernels' adjoint always reads transforms: without the cache it recomputes them
    // into the same buffer first)
    p->cache_on = p->phi && !((prm.precision > 0 || cl) && prm.phi_cache == 0);
    if (!rc && prm.precision > 0) {
        rc = dalloc(p, &p->tc_ops, (size_t)kTcOps * kTcOpBytes);
        if (!rc) {
            k_tc_ops<<<kTcOps, 256>>>(reinterpret_cast<unsigned short *>(p->tc_ops));
            if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = QST_ERR_CUDA;
        }
    }
    if (!rc) rc = dalloc(p, &p->it_state, 1);
    if (!rc && cudaMemset(p->it_state, 0, sizeof(IterState)) != cudaSuccess) rc = QST_ERR_CUDA;
    if (!rc) rc = dalloc(p, &p->it_c, nnz);
    if (!rc) {
        std::vector<float> m1((size_t)K, -1.0f);
        if (cudaMemcpy(p->step_m1, m1.data(), sizeof(float) * K, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = QST_ERR_CUDA;
    }
    if (!rc) rc = dalloc(p, &p->status, 1);
    if (!rc && cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) rc = QST_ERR_CUDA;
    if (!rc) {
        with_geo(p->c, p->A, [](auto cc, auto ra) { set_smem_attrs<decltype(cc)::value, decltype(ra)::value>(); });
        if (p->fx) {
            cudaFuncSetAttribute(k_forward_fx, cudaFuncAttributeMaxDynamicSharedMemorySize, fx_smem(false).total);
            cudaFuncSetAttribute(k_adjoint_fx, cudaFuncAttributeMaxDynamicSharedMemorySize, fx_smem(true).total);
        }
        if (p->wide) {
            cudaFuncSetAttribute(k_forward_fx1p<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFx1pFwdSmem);
            cudaFuncSetAttribute(k_forward_fx1p<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFx1pFwdSmem);
            cudaFuncSetAttribute(k_adjoint_fx1p, cudaFuncAttributeMaxDynamicSharedMemorySize, kFx1pAdjSmem);
            cudaFuncSetAttribute(k_adjoint_fx1cp, cudaFuncAttributeMaxDynamicSharedMemorySize, kFx1pAdjcSmem);
            cudaFuncSetAttribute(k_high_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kWideSmem);
            cudaFuncSetAttribute(k_high_inv_acc, cudaFuncAttributeMaxDynamicSharedMemorySize, kWideInvSmem);
        }
        if (p->cl) {
            cudaFuncSetAttribute(k_forward_cl<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cl_smem().total);
            cudaFuncSetAttribute(k_forward_cl<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cl_smem().total);
            cudaFuncSetAttribute(k_adjoint_clc, cudaFuncAttributeMaxDynamicSharedMemorySize, cl_smem().total);
        }
        if (p->fx2) {
            cudaFuncSetAttribute(k_forward_2r<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
            cudaFuncSetAttribute(k_forward_2r<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
            cudaFuncSetAttribute(k_adjoint_2c<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2c_smem(k2cStageSingle).total);
            cudaFuncSetAttribute(k_adjoint_2c<11>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2c_smem(k2cStageSingle).total);
            cudaFuncSetAttribute(k_adjoint_2c<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2c_smem(k2cStageSingle).total);
            cudaFuncSetAttribute(k_forward_2r<false, 11>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
            cudaFuncSetAttribute(k_forward_2r<true, 11>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
            cudaFuncSetAttribute(k_forward_2r<false, 10>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
            cudaFuncSetAttribute(k_forward_2r<true, 10>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
            cudaFuncSetAttribute(k_adjoint_2r<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2p_smem().total);
            cudaFuncSetAttribute(k_adjoint_2r<11>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2p_smem().total);
            cudaFuncSetAttribute(k_adjoint_2r<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2p_smem().total);
        }
        if (prm.precision > 0) {
            cudaFuncSetAttribute(k_forward_tc<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemAlloc);
            cudaFuncSetAttribute(k_forward_tc<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemAlloc);
            cudaFuncSetAttribute(k_forward_tc<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemAlloc);
            cudaFuncSetAttribute(k_forward_tc<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemAlloc);
            cudaFuncSetAttribute(k_forward_tc<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemAlloc);
            cudaFuncSetAttribute(k_forward_tc<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemAlloc);
            cudaFuncSetAttribute(k_adjoint_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemAlloc);
            cudaFuncSetAttribute(k_adjoint_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemAlloc);
            cudaFuncSetAttribute(k_adjoint_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemAlloc);
        }
        if (cudaGetLastError() != cudaSuccess) rc = QST_ERR_CUDA;
    }
    if (rc) {
        qst_plan_destroy(p);
        return rc;
    }
    *out = p;
    return QST_OK;
}

qst_status qst_plan_destroy(qst_plan p) {
    if (!p) return QST_ERR_INVALID_ARG;
    cudaFree(p->phi);
    cudaFree(p->tc_ops);
    cudaFree(p->it_Jseg);
    cudaFree(p->it_aseg);
    cudaFree(p->plans);
    cudaFree(p->order);
    cudaFree(p->bins);
    cudaFree(p->n_bins);
    cudaFree(p->choff);
    cudaFree(p->ppart);
    cudaFree(p->loss_part);
    if (!p->wide) cudaFree(p->zbuf);
    cudaFree(p->wide_T);
    cudaFree(p->wide_acc);
    cudaFree(p->cl_perm);
    cudaFree(p->cl_pu);
    cudaFree(p->cl_ofs);
    cudaFree(p->hdot);
    cudaFree(p->refac_C);
    cudaFree(p->refac_T);
    cudaFree(p->step_trial);
    cudaFree(p->step_grad);
    cudaFree(p->step_c);
    cudaFree(p->step_gw);
    cudaFree(p->step_tw);
    cudaFree(p->step_m1);
    cudaFree(p->step_loss);
    cudaFree(p->step_kout);
    cudaFree(p->status);
    cudaFree(p->h_dev);
    if (p->h_side) cudaStreamDestroy(p->h_side);
    if (p->h_fork) cudaEventDestroy(p->h_fork);
    if (p->h_count) cudaEventDestroy(p->h_count);
    cudaFree(p->it_state);
    cudaFree(p->it_c);
    for (void *q : {(void *)p->lz_Q, (void *)p->lz_SQ, (void *)p->lz_W, (void *)p->lz_C, (void *)p->lz_P,
                    (void *)p->lz_G, (void *)p->lz_Tm, (void *)p->lz_T, (void *)p->lz_Y, (void *)p->lz_Tc,
                    (void *)p->lz_lam, (void *)p->lz_int})
        cudaFree(q);
    if (p->it_exec) cudaGraphExecDestroy(p->it_exec);
    if (p->it_cap) cudaStreamDestroy(p->it_cap);
    if (p->it_body) cudaStreamDestroy(p->it_body);
    for (auto &tl : p->pending) {
        cudaEventDestroy(tl.start);
        cudaEventDestroy(tl.stop);
    }
    for (auto e : p->pool) cudaEventDestroy(e);
    delete p;
    return QST_OK;
}

qst_status qst_plan_workspace_bytes(qst_plan p, int64_t *bytes) {
    if (!p || !bytes) return QST_ERR_INVALID_ARG;
    *bytes = p->ws_bytes;
    return QST_OK;
}

qst_status qst_tangent(qst_plan p, const float *psi, const float *w, const float *grad_psi, const float *grad_w,
                       float *d, void *stream) {
    if (!p || !psi || !w || !grad_psi || !grad_w || !d) return QST_ERR_INVALID_ARG;
    if (!aligned(psi, 8) || !aligned(grad_psi, 8) || !aligned(d, 8) || !aligned(w, 4) || !aligned(grad_w, 4))
        return QST_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t total = (int64_t)p->K << p->n;
    return launch(p, QST_KERNEL_TANGENT, st, [&] {
        k_tangent<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            reinterpret_cast<const float2 *>(psi), w, reinterpret_cast<const float2 *>(grad_psi), grad_w,
            reinterpret_cast<float2 *>(d), p->n, p->K);
    });
}

qst_status qst_plan_geometry(qst_plan p, int *chunk_qubits, int *high_qubits, int *fixed_rounds) {
    if (!p) return QST_ERR_INVALID_ARG;
    if (chunk_qubits) *chunk_qubits = p->c;
    if (high_qubits) *high_qubits = p->r;
    if (fixed_rounds) *fixed_rounds = p->cl ? 4 : (p->fw ? 3 : (p->fx2 ? 2 : (p->fx ? 1 : 0)));
    return QST_OK;
}

qst_status qst_forward(qst_plan p, const float *psi, const float *w, const uint8_t *basis, const int64_t *row_ptr,
                       const uint32_t *outcome, const uint32_t *count, const uint32_t *shots, float *p_obs,
                       float *c_obs, double *loss, float *p_dense, void *stream) {
    if (!p || !psi || !w || !basis || !row_ptr || !shots) return QST_ERR_INVALID_ARG;
    if (p->nnz > 0 && (!outcome || !count)) return QST_ERR_INVALID_ARG;
    if (!aligned(psi, 16) || !aligned(w, 4) || !aligned(row_ptr, 8) || (outcome && !aligned(outcome, 4)) ||
        (count && !aligned(count, 4)) || !aligned(shots, 4) || (p_obs && !aligned(p_obs, 4)) ||
        (c_obs && !aligned(c_obs, 4)) || (loss && !aligned(loss, 8)) || (p_dense && !aligned(p_dense, 4)))
        return QST_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    qst_status rc = prepare(p, basis, row_ptr, outcome, shots, st);
    if (rc) return rc;
    return forward_core(p, psi, w, row_ptr, outcome, count, shots, p_obs, c_obs, loss, p_dense, nullptr, st);
}

}  // extern "C"

namespace {
// The forward after packing and validation; with `skip` set on the device
// (optional) every launch returns at once.
qst_status forward_core(qst_plan p, const float *psi, const float *w, const int64_t *row_ptr, const uint32_t *outcome,
                        const uint32_t *count, const uint32_t *shots, float *p_obs, float *c_obs, double *loss,
                        float *p_dense, const int *skip, cudaStream_t st, float2 *phi_cache,
                        cudaEvent_t count_ready) {
    qst_status rc = QST_OK;
    if (p_dense && cudaMemsetAsync(p_dense, 0, (size_t)p->M * ((size_t)1 << p->n) * sizeof(float), st) != cudaSuccess)
        return QST_ERR_CUDA;
    if (p->wide) {
        rc = forward_wide(p, reinterpret_cast<const float2 *>(psi), w, row_ptr, outcome, p_dense, st, phi_cache);
        if (rc) return rc;
    }
    FwdArgs a;
    a.psi = reinterpret_cast<const float2 *>(psi);
    a.w = w;
    a.plans = p->plans;
    a.order = p->order;
    a.bins = p->bins;
    a.n_bins = p->n_bins;
    a.row_ptr = row_ptr;
    a.outcome = outcome;
    a.choff = p->choff;
    a.ppart = p->ppart;
    a.p_dense = p_dense;
    a.nnz = p->nnz;
    a.n = p->n;
    a.r = p->r;
    a.K = p->K;
    a.src_bin_stride = 0;
    a.skip = skip;
    a.phi_obs = phi_cache;
    const int units = p->nb_max << p->r;
    if (!p->wide) {
        rc = launch(p, QST_KERNEL_FORWARD, st, [&] {
            launch_forward_units(p, a, units, st);
        });
        if (rc) return rc;
    }
    // the counts are first read by the epilogue: their copy may still be in flight until here
    if (count_ready && cudaStreamWaitEvent(st, count_ready, 0) != cudaSuccess) return QST_ERR_CUDA;
    const float invB = 1.0f / (float)p->B;
    const int egrid = p->loss_parts;
    rc = launch(p, QST_KERNEL_EPILOGUE, st, [&] {
        k_fwd_epilogue<<<egrid, 256, 0, st>>>(p->ppart, row_ptr, count, shots, p->M, p->K, p->nnz, invB,
                                              (float)p->prm.eps, p_obs, c_obs, p->loss_part, skip);
    });
    if (rc) return rc;
    return launch(p, QST_KERNEL_LOSS, st, [&] {
        k_loss<<<1, 256, 0, st>>>(p->loss_part, p->loss_parts, loss, p->status, skip);
    });
}
}  // namespace

extern "C" {

qst_status qst_adjoint(qst_plan p, const float *psi, const float *w, const uint8_t *basis, const int64_t *row_ptr,
                       const uint32_t *outcome, const float *c_obs, float *grad_psi, float *grad_w, void *stream) {
    if (!p || !psi || !w || !basis || !row_ptr || !grad_psi) return QST_ERR_INVALID_ARG;
    if (p->nnz > 0 && (!outcome || !c_obs)) return QST_ERR_INVALID_ARG;
    if (!aligned(psi, 16) || !aligned(grad_psi, 16) || !aligned(w, 4) || !aligned(row_ptr, 8) ||
        (outcome && !aligned(outcome, 4)) || (c_obs && !aligned(c_obs, 4)) || (grad_w && !aligned(grad_w, 4)))
        return QST_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // shots are only validated in the forward; the adjoint reads c directly
    qst_status rc = prepare(p, basis, row_ptr, outcome, nullptr, st);
    if (rc) return rc;
    return adjoint_core(p, psi, w, row_ptr, outcome, c_obs, grad_psi, grad_w, st);
}

}  // extern "C"

namespace {
// The adjoint after packing and validation.
qst_status adjoint_core(qst_plan p, const float *psi, const float *w, const int64_t *row_ptr, const uint32_t *outcome,
                        const float *c_obs, float *grad_psi, float *grad_w, cudaStream_t st,
                        const float2 *phi_cache, const int *skip) {
    qst_status rc = QST_OK;
    AdjArgs a;
    a.psi = reinterpret_cast<const float2 *>(psi);
    a.plans = p->plans;
    a.order = p->order;
    a.bins = p->bins;
    a.n_bins = p->n_bins;
    a.row_ptr = row_ptr;
    a.outcome = outcome;
    a.c_obs = c_obs;
    a.choff = p->choff;
    a.zbuf = p->zbuf;
    a.n = p->n;
    a.r = p->r;
    a.K = p->K;
    a.src_bin_stride = 0;
    a.phi_obs = phi_cache;
    a.nnz = p->nnz;
    a.skip = skip;
    if (p->wide) {
        rc = adjoint_wide(p, reinterpret_cast<const float2 *>(psi), w, row_ptr, outcome, c_obs,
                          reinterpret_cast<float2 *>(grad_psi), st, phi_cache);
        if (rc || !grad_w) return rc;
        const float invBw = 1.0f / (float)p->B;
        return launch(p, QST_KERNEL_HSUM, st, [&] { k_hsum<<<p->K, 256, 0, st>>>(p->hdot, p->c, invBw, grad_w, nullptr); });
    }
    const int units = p->nb_max << p->r;
    if (((p->fx2 && p->prm.precision > 0) || p->cl) && !phi_cache) {
        // the tensor-core and cluster adjoints read transforms: recompute them with the plan's
        // forward (its w |.|^2 partials go to the plan's scratch and are not read)
        FwdArgs f;
        f.psi = a.psi;
        f.w = w;
        f.plans = p->plans;
        f.order = p->order;
        f.bins = p->bins;
        f.n_bins = p->n_bins;
        f.row_ptr = row_ptr;
        f.outcome = outcome;
        f.choff = p->choff;
        f.ppart = p->ppart;
        f.p_dense = nullptr;
        f.nnz = p->nnz;
        f.src_bin_stride = 0;
        f.skip = skip;
        f.n = p->n;
        f.r = p->r;
        f.K = p->K;
        f.phi_obs = p->phi;
        rc = launch(p, QST_KERNEL_FORWARD, st, [&] { launch_forward_units(p, f, units, st); });
        if (rc) return rc;
        a.phi_obs = p->phi;
    }
    rc = launch(p, QST_KERNEL_ADJOINT, st, [&] {
        launch_adjoint_units(p, a, units, st);
    });
    if (rc) return rc;
    const float invB = 1.0f / (float)p->B;
    const int64_t total = (int64_t)p->K << p->c;
    const int rgrid = (int)((total + 255) / 256);
    float2 *g = reinterpret_cast<float2 *>(grad_psi);
    rc = launch(p, QST_KERNEL_REDUCE, st, [&] {
        switch (p->r) {
            case 0: k_reduce<0><<<rgrid, 256, 0, st>>>(p->zbuf, p->bins, p->n_bins, w, reinterpret_cast<const float2 *>(psi), g, p->hdot, p->n, p->c, p->K, invB, skip); break;
            case 1: k_reduce<1><<<rgrid, 256, 0, st>>>(p->zbuf, p->bins, p->n_bins, w, reinterpret_cast<const float2 *>(psi), g, p->hdot, p->n, p->c, p->K, invB, skip); break;
            case 2: k_reduce<2><<<rgrid, 256, 0, st>>>(p->zbuf, p->bins, p->n_bins, w, reinterpret_cast<const float2 *>(psi), g, p->hdot, p->n, p->c, p->K, invB, skip); break;
            case 3: k_reduce<3><<<rgrid, 256, 0, st>>>(p->zbuf, p->bins, p->n_bins, w, reinterpret_cast<const float2 *>(psi), g, p->hdot, p->n, p->c, p->K, invB, skip); break;
            default: k_reduce<4><<<rgrid, 256, 0, st>>>(p->zbuf, p->bins, p->n_bins, w, reinterpret_cast<const float2 *>(psi), g, p->hdot, p->n, p->c, p->K, invB, skip); break;
        }
    });
    if (rc || !grad_w) return rc;
    return launch(p, QST_KERNEL_HSUM, st, [&] {
        k_hsum<<<p->K, 256, 0, st>>>(p->hdot, p->c, invB, grad_w, skip);
    });
}
}  // namespace

extern "C" {

qst_status qst_evaluate(qst_plan p, const float *psi, const float *w, const uint8_t *basis, const int64_t *row_ptr,
                        const uint32_t *outcome, const uint32_t *count, const uint32_t *shots, float *p_obs,
                        float *c_obs, double *loss, float *grad_psi, float *grad_w, void *stream) {
    if (!p || !psi || !w || !basis || !row_ptr || !shots || !c_obs || !grad_psi) return QST_ERR_INVALID_ARG;
    if (p->nnz > 0 && (!outcome || !count)) return QST_ERR_INVALID_ARG;
    if (!aligned(psi, 16) || !aligned(grad_psi, 16) || !aligned(w, 4) || !aligned(row_ptr, 8) ||
        (outcome && !aligned(outcome, 4)) || (count && !aligned(count, 4)) || !aligned(shots, 4) ||
        (p_obs && !aligned(p_obs, 4)) || !aligned(c_obs, 4) || (loss && !aligned(loss, 8)) ||
        (grad_w && !aligned(grad_w, 4)))
        return QST_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    qst_status rc = prepare(p, basis, row_ptr, outcome, shots, st);
    if (!rc) rc = forward_core(p, psi, w, row_ptr, outcome, count, shots, p_obs, c_obs, loss, nullptr, nullptr, st,
                               p->cache_on ? p->phi : nullptr);
    if (!rc) rc = adjoint_core(p, psi, w, row_ptr, outcome, c_obs, grad_psi, grad_w, st, p->cache_on ? p->phi : nullptr);
    return rc;
}

qst_status qst_evaluate_host(qst_plan p, const float *psi, const float *w, const uint8_t *basis,
                             const int64_t *row_ptr, const uint32_t *outcome, const uint32_t *count,
                             const uint32_t *shots, double *loss_out, float *grad_psi_out, float *grad_w_out,
                             float *c_obs_out, void *stream) {
    if (!p || !psi || !w || !basis || !row_ptr || !shots || !loss_out || !grad_psi_out || !grad_w_out)
        return QST_ERR_INVALID_ARG;
    if (p->nnz > 0 && (!outcome || !count)) return QST_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t D = (size_t)1 << p->n;
    const size_t b_psi = (size_t)p->K * D * 8, b_w = (size_t)p->K * 4, b_basis = (size_t)p->M * p->n;
    const size_t b_row = (size_t)(p->M + 1) * 8, b_nnz = (size_t)p->nnz * 4, b_shots = (size_t)p->M * 4;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_psi = 0, o_grad = o_psi + up(b_psi), o_w = o_grad + up(b_psi), o_gw = o_w + up(b_w),
                 o_row = o_gw + up(b_w), o_out = o_row + up(b_row), o_cnt = o_out + up(b_nnz),
                 o_c = o_cnt + up(b_nnz), o_shots = o_c + up(b_nnz), o_basis = o_shots + up(b_shots),
                 o_loss = o_basis + up(b_basis), total = o_loss + 256;
    if (!p->h_dev) {
        if (cudaMalloc(&p->h_dev, total) != cudaSuccess) {
            cudaGetLastError();
            return QST_ERR_NO_MEMORY;
        }
        p->ws_bytes += (int64_t)total;
    }
    char *base = (char *)p->h_dev;
#define QST_H2D(off, src, bytes)                                                                   \
    if ((bytes) && cudaMemcpyAsync(base + (off), (src), (bytes), cudaMemcpyHostToDevice, st) != cudaSuccess) \
        return QST_ERR_CUDA;
    QST_H2D(o_psi, psi, b_psi);
    QST_H2D(o_w, w, b_w);
    QST_H2D(o_basis, basis, b_basis);
    QST_H2D(o_row, row_ptr, b_row);
    QST_H2D(o_out, outcome, b_nnz);
    QST_H2D(o_shots, shots, b_shots);
#undef QST_H2D
    // the counts (read first by the forward's epilogue) are copied on a side stream while
    // the packing, the validation and the forward chunk kernels run
    if (!p->h_side && (cudaStreamCreateWithFlags(&p->h_side, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaEventCreateWithFlags(&p->h_fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&p->h_count, cudaEventDisableTiming) != cudaSuccess))
        return QST_ERR_CUDA;
    if (cudaEventRecord(p->h_fork, st) != cudaSuccess || cudaStreamWaitEvent(p->h_side, p->h_fork, 0) != cudaSuccess)
        return QST_ERR_CUDA;
    if (b_nnz && cudaMemcpyAsync(base + o_cnt, count, b_nnz, cudaMemcpyHostToDevice, p->h_side) != cudaSuccess)
        return QST_ERR_CUDA;
    if (cudaEventRecord(p->h_count, p->h_side) != cudaSuccess) return QST_ERR_CUDA;
    const float *d_psi = (const float *)(base + o_psi);
    const float *d_w = (const float *)(base + o_w);
    const int64_t *d_row = (const int64_t *)(base + o_row);
    const uint32_t *d_out = (const uint32_t *)(base + o_out);
    qst_status rc = prepare(p, (const uint8_t *)(base + o_basis), d_row, d_out, (const uint32_t *)(base + o_shots), st);
    if (!rc) rc = forward_core(p, d_psi, d_w, d_row, d_out, (const uint32_t *)(base + o_cnt),
                               (const uint32_t *)(base + o_shots), nullptr, (float *)(base + o_c),
                               (double *)(base + o_loss), nullptr, nullptr, st, p->cache_on ? p->phi : nullptr,
                               p->h_count);
    if (!rc) rc = adjoint_core(p, d_psi, d_w, d_row, d_out, (const float *)(base + o_c), (float *)(base + o_grad),
                               (float *)(base + o_gw), st, p->cache_on ? p->phi : nullptr);
    if (rc) {
        cudaStreamSynchronize(p->h_side);
        return rc;
    }
    if (cudaMemcpyAsync(loss_out, base + o_loss, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return QST_ERR_CUDA;
    if (cudaMemcpyAsync(grad_psi_out, base + o_grad, b_psi, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return QST_ERR_CUDA;
    if (cudaMemcpyAsync(grad_w_out, base + o_gw, b_w, cudaMemcpyDeviceToHost, st) != cudaSuccess) return QST_ERR_CUDA;
    if (c_obs_out && b_nnz &&
        cudaMemcpyAsync(c_obs_out, base + o_c, b_nnz, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return QST_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return QST_ERR_CUDA;
    return QST_OK;
}

qst_status qst_plan_status(qst_plan p, int *device_status) {
    if (!p) return QST_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return QST_ERR_CUDA;
    int st = 0;
    if (cudaMemcpy(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return QST_ERR_CUDA;
    if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) return QST_ERR_CUDA;
    if (device_status) *device_status = st;
    return st ? QST_ERR_DEVICE : QST_OK;
}

qst_status qst_plan_set_timing(qst_plan p, int enable) {
    if (!p) return QST_ERR_INVALID_ARG;
    p->timing = enable != 0;
    return QST_OK;
}

qst_status qst_plan_kernel_stats(qst_plan p, int64_t *launches, double *ms, int kinds) {
    if (!p || kinds < 0) return QST_ERR_INVALID_ARG;
    resolve_pending(p);
    for (int i = 0; i < kinds && i < QST_KERNEL_KINDS; ++i) {
        if (launches) launches[i] = p->launches[i];
        if (ms) ms[i] = p->ms[i];
    }
    return QST_OK;
}

qst_status qst_plan_reset_stats(qst_plan p) {
    if (!p) return QST_ERR_INVALID_ARG;
    resolve_pending(p);
    for (int i = 0; i < QST_KERNEL_KINDS; ++i) {
        p->launches[i] = 0;
        p->ms[i] = 0.0;
    }
    p->total_launches = 0;
    return QST_OK;
}

qst_status qst_plan_launch_count(qst_plan p, int64_t *count) {
    if (!p || !count) return QST_ERR_INVALID_ARG;
    *count = p->total_launches;
    return QST_OK;
}

qst_status qst_simplex_project(const double *v, int K, double tau, double *beta, int *keep, int *K_out,
                               void *stream) {
    if (!v || !beta || !keep || !K_out || K < 1) return QST_ERR_INVALID_ARG;
    if (K > kProjMax) return QST_ERR_UNSUPPORTED;
    if (!aligned(v, 8) || !aligned(beta, 8) || !aligned(keep, 4) || !aligned(K_out, 4)) return QST_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    k_simplex<<<1, kProjMax, 0, st>>>(v, K, tau, beta, keep, K_out);
    return cudaGetLastError() == cudaSuccess ? QST_OK : QST_ERR_CUDA;
}

}  // extern "C"

namespace {
// The spectral step's proposal for one eta (Sec. III-C): block Krylov basis of
// S = Psi diag(w) Psi^* + eta G started at the atoms, Rayleigh-Ritz, candidates,
// selection.  Writes the proposal's atoms (K rows; zero beyond the kept count)
// and weights.  G uses the likelihood ratio of the current state in
// p->step_c.  Synchronises to read the size of each orthonormalised block.
qst_status spectral_candidate(qst_plan p, const float *psi, const float *w, const int64_t *row_ptr,
                              const uint32_t *outcome, double eta, const qst_step_params &sp, float2 *trial,
                              float *tw, cudaStream_t st) {
    const int K = p->K;
    const int64_t D = (int64_t)1 << p->n;
    const size_t vb = sizeof(float2) * (size_t)D;
    const float2 *ps = reinterpret_cast<const float2 *>(psi);
    const int cgrid = (int)((D + 255) / 256 < 148 * 8 ? (D + 255) / 256 : 148 * 8);
    constexpr double kDrop = 1e-10;
    qst_status rc = QST_OK;
    auto read_int = [&](int *h) -> qst_status {
        if (cudaMemcpyAsync(h, p->lz_int, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return QST_ERR_CUDA;
        return QST_OK;
    };
    // W (kb rows) -> orthonormal rows in place (kept first); P: its Gram matrix before projections
    auto orth = [&](int kb, const double2 *P, int *kept) -> qst_status {
        qst_status r2 = launch(p, QST_KERNEL_STEP, st, [&] {
            k_xgram<<<kb * kb, 256, 0, st>>>(p->lz_W, kb, p->lz_W, kb, D, p->lz_G, kb);
        });
        if (!r2) r2 = launch(p, QST_KERNEL_STEP, st, [&] {
            k_orth_coef<<<1, kRefacMax, 0, st>>>(p->lz_G, P, kb, kDrop, p->lz_Tm, p->lz_int);
        });
        if (!r2) r2 = launch(p, QST_KERNEL_STEP, st, [&] { k_combine<<<cgrid, 256, 0, st>>>(p->lz_W, kb, D, p->lz_Tm); });
        if (!r2) r2 = read_int(kept);
        return r2;
    };
    // block 0: the atoms
    if (cudaMemcpyAsync(p->lz_W, psi, vb * K, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return QST_ERR_CUDA;
    rc = launch(p, QST_KERNEL_STEP, st, [&] { k_xgram<<<K * K, 256, 0, st>>>(ps, K, ps, K, D, p->lz_P, K); });
    int kb = 0;
    if (!rc) rc = orth(K, p->lz_P, &kb);
    if (rc) return rc;
    int m = 0, mb = 0;
    if (kb > 0 && cudaMemcpyAsync(p->lz_Q, p->lz_W, vb * kb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return QST_ERR_CUDA;
    m = kb;
    p->lz_blocks = 0;
    while (kb > 0) {
        // SQ_block = eta G Q_block + Psi diag(w) (Psi^* Q_block); the adjoint takes K rows, zero beyond kb
        float2 *qb = p->lz_Q + (size_t)mb * D, *sq = p->lz_SQ + (size_t)mb * D;
        if (kb < K && cudaMemsetAsync(p->lz_Q + (size_t)m * D, 0, vb * (K - kb), st) != cudaSuccess) return QST_ERR_CUDA;
        rc = adjoint_core(p, reinterpret_cast<const float *>(qb), p->step_m1, row_ptr, outcome, p->step_c,
                          reinterpret_cast<float *>(sq), nullptr, st);
        p->lz_blocks += 1;
        if (!rc) rc = launch(p, QST_KERNEL_STEP, st, [&] {
            k_xgram<<<K * kb, 256, 0, st>>>(ps, K, qb, kb, D, p->lz_C, kb);
        });
        if (!rc) rc = launch(p, QST_KERNEL_STEP, st, [&] {
            k_lincomb<<<cgrid, 256, 0, st>>>(sq, kb, eta, ps, K, p->lz_C, kb, w, 1.0, D);
        });
        if (rc) return rc;
        if (m + K > sp.n_krylov) break;
        // W = SQ_block minus its components on the basis, twice; then orthonormalise
        if (cudaMemcpyAsync(p->lz_W, sq, vb * kb, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return QST_ERR_CUDA;
        rc = launch(p, QST_KERNEL_STEP, st, [&] {
            k_xgram<<<kb * kb, 256, 0, st>>>(p->lz_W, kb, p->lz_W, kb, D, p->lz_P, kb);
        });
        for (int pass = 0; pass < 2 && !rc; ++pass) {
            rc = launch(p, QST_KERNEL_STEP, st, [&] {
                k_xgram<<<m * kb, 256, 0, st>>>(p->lz_Q, m, p->lz_W, kb, D, p->lz_C, kb);
            });
            if (!rc) rc = launch(p, QST_KERNEL_STEP, st, [&] {
                k_lincomb<<<cgrid, 256, 0, st>>>(p->lz_W, kb, 1.0, p->lz_Q, m, p->lz_C, kb, nullptr, -1.0, D);
            });
        }
        int kn = 0;
        if (!rc) rc = orth(kb, p->lz_P, &kn);
        if (rc) return rc;
        if (kn == 0) break;
        if (cudaMemcpyAsync(p->lz_Q + (size_t)m * D, p->lz_W, vb * kn, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return QST_ERR_CUDA;
        mb = m;
        kb = kn;
        m += kn;
    }
    if (m == 0) return QST_ERR_INVALID_ARG;  // every atom is zero
    // Rayleigh-Ritz and the candidates
    rc = launch(p, QST_KERNEL_STEP, st, [&] {
        k_xgram<<<m * m, 256, 0, st>>>(p->lz_Q, m, p->lz_SQ, m, D, p->lz_T, m);
    });
    if (!rc) rc = launch(p, QST_KERNEL_STEP, st, [&] { k_heig<<<1, kRefacMax, 0, st>>>(p->lz_T, m, p->lz_lam, p->lz_Y); });
    const int L = K < m ? K : m;
    if (!rc) rc = launch(p, QST_KERNEL_STEP, st, [&] {
        k_spectral_select<<<1, 32, 0, st>>>(p->lz_lam, p->lz_Y, m, L, eta, sp.mu, sp.tau, K, p->lz_Tc, tw, p->lz_int,
                                            p->lz_int + 1, sp.rank_fix);
    });
    if (!rc && cudaMemsetAsync(trial, 0, vb * K, st) != cudaSuccess) rc = QST_ERR_CUDA;
    if (!rc) rc = launch(p, QST_KERNEL_STEP, st, [&] {
        k_lincomb<<<cgrid, 256, 0, st>>>(trial, K, 0.0, p->lz_Q, m, p->lz_Tc, K, nullptr, 1.0, D);
    });
    return rc;
}
}  // namespace

extern "C" {

void qst_step_params_default(qst_step_params *sp) {
    if (!sp) return;
    sp->mu = 1e-3;
    sp->tau = 1e-3;
    sp->tau_acc = 1e-10;
    sp->eta0 = 1.0;
    sp->eta_ratio = 0.5;
    sp->n_eta = 11;
    sp->n_krylov = 30;
    sp->rank_fix = 0;
}

qst_status qst_step(qst_plan p, int slot, int r, float *psi, float *w, const uint8_t *basis, const int64_t *row_ptr,
                    const uint32_t *outcome, const uint32_t *count, const uint32_t *shots,
                    const qst_step_params *params, double *J_out, int *accepted, double *eta_used, void *stream) {
    if (!p || !psi || !w || !basis || !row_ptr || !shots || !J_out || !accepted || !eta_used) return QST_ERR_INVALID_ARG;
    if (slot < 0 || slot > 3 || (slot == 0 && (r < 0 || r >= p->K))) return QST_ERR_INVALID_ARG;
    if (p->K > kProjMax || (slot == 2 && !p->refac_C) || (slot == 3 && !p->lz_Q)) return QST_ERR_UNSUPPORTED;
    qst_step_params sp;
    qst_step_params_default(&sp);
    if (params) sp = *params;
    if (sp.n_eta < 1 || !(sp.eta0 > 0.0) || !(sp.eta_ratio > 0.0)) return QST_ERR_INVALID_ARG;
    if (slot == 3 && (sp.n_krylov < 2 * p->K || sp.n_krylov > kKrylovMax)) return QST_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int K = p->K;
    const size_t D = (size_t)1 << p->n;
    std::vector<float> wh((size_t)K);
    // J = L_eps + mu R for the state (ps, ww); R counts the atoms with w > 0.
    int R_last = 0;  // active atoms of the last evaluated state
    auto evaluate = [&](const float *ps, const float *ww, float *c_out, double *J) -> qst_status {
        qst_status rc = qst_forward(p, ps, ww, basis, row_ptr, outcome, count, shots, nullptr, c_out, p->step_loss,
                                    nullptr, stream);
        if (rc) return rc;
        double L = 0.0;
        if (cudaMemcpyAsync(&L, p->step_loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(wh.data(), ww, sizeof(float) * K, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return QST_ERR_CUDA;
        int R = 0;
        for (int k = 0; k < K; ++k) R += wh[k] > 0.f;
        R_last = R;
        *J = L + sp.mu * R;
        return QST_OK;
    };
    double J0 = 0.0;
    qst_status rc = evaluate(psi, w, p->step_c, &J0);
    if (rc) return rc;
    *J_out = J0;
    *accepted = 0;
    *eta_used = 0.0;
    float *trial_psi = reinterpret_cast<float *>(p->step_trial);
    if (slot == 2) {  // exact spectral refactorisation (eta_rho = 0)
        if (cudaMemcpyAsync(trial_psi, psi, sizeof(float2) * K * D, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(p->step_tw, w, sizeof(float) * K, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return QST_ERR_CUDA;
        rc = qst_refactor(p, trial_psi, p->step_tw, sp.tau, p->step_kout, stream);
        if (rc) return rc;
        double Jt = 0.0;
        rc = evaluate(trial_psi, p->step_tw, nullptr, &Jt);
        if (rc) return rc;
        if (Jt <= J0 - sp.tau_acc) {
            if (cudaMemcpyAsync(psi, trial_psi, sizeof(float2) * K * D, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaMemcpyAsync(w, p->step_tw, sizeof(float) * K, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return QST_ERR_CUDA;
            *J_out = Jt;
            *accepted = 1;
        }
        return QST_OK;
    }
    double eta = sp.eta0;
    if (slot == 3) {  // spectral step (Sec. III-C) with eta_rho on the step grid
        // serial-equivalent oracle calls per trial: G on every Krylov block (K vectors), the new
        // atoms' responses and the loss
        p->step_calls = 0;
        for (int j = 0; j < sp.n_eta; ++j, eta *= sp.eta_ratio) {
            rc = spectral_candidate(p, psi, w, row_ptr, outcome, eta, sp, p->step_trial, p->step_tw, st);
            if (rc) return rc;
            double Jt = 0.0;
            rc = evaluate(trial_psi, p->step_tw, nullptr, &Jt);
            if (rc) return rc;
            p->step_calls += (long long)p->lz_blocks * K + R_last + 1;
            if (Jt <= J0 - sp.tau_acc) {
                if (cudaMemcpyAsync(psi, trial_psi, sizeof(float2) * K * D, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                    cudaMemcpyAsync(w, p->step_tw, sizeof(float) * K, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess)
                    return QST_ERR_CUDA;
                *J_out = Jt;
                *accepted = 1;
                *eta_used = eta;
                return QST_OK;
            }
        }
        *eta_used = eta / sp.eta_ratio;
        return QST_OK;
    }
    if (slot == 0) {  // atom r (Eqs. atom-direction, atom-trial)
        rc = qst_adjoint(p, psi, p->step_m1, basis, row_ptr, outcome, p->step_c,
                         reinterpret_cast<float *>(p->step_grad), nullptr, stream);
        if (rc) return rc;
        if (cudaMemcpyAsync(trial_psi, psi, sizeof(float2) * K * D, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return QST_ERR_CUDA;
        float2 *out = p->step_trial + (size_t)r * D;
        for (int j = 0; j < sp.n_eta; ++j, eta *= sp.eta_ratio) {
            rc = launch(p, QST_KERNEL_STEP, st, [&] {
                k_atom_trial<<<1, 1024, 0, st>>>(reinterpret_cast<const float2 *>(psi), p->step_grad, w, nullptr, r,
                                                 eta, (int64_t)D, p->step_trial, nullptr);
            });
            if (rc) return rc;
            double Jt = 0.0;
            rc = evaluate(trial_psi, w, nullptr, &Jt);
            if (rc) return rc;
            if (Jt <= J0 - sp.tau_acc) {
                if (cudaMemcpyAsync(reinterpret_cast<float2 *>(psi) + (size_t)r * D, out, sizeof(float2) * D,
                                    cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess)
                    return QST_ERR_CUDA;
                *J_out = Jt;
                *accepted = 1;
                *eta_used = eta;
                return QST_OK;
            }
        }
        *eta_used = eta / sp.eta_ratio;
        return QST_OK;
    }
    // slot 1: coefficients (Eq. coefficient-update, then P_tau)
    rc = qst_adjoint(p, psi, w, basis, row_ptr, outcome, p->step_c, reinterpret_cast<float *>(p->step_grad),
                     p->step_gw, stream);
    if (rc) return rc;
    for (int j = 0; j < sp.n_eta; ++j, eta *= sp.eta_ratio) {
        rc = launch(p, QST_KERNEL_STEP, st, [&] {
            k_coeff_trial<<<1, kProjMax, 0, st>>>(w, p->step_gw, eta, sp.tau, K, p->step_tw, nullptr);
        });
        if (rc) return rc;
        double Jt = 0.0;
        rc = evaluate(psi, p->step_tw, nullptr, &Jt);
        if (rc) return rc;
        if (Jt <= J0 - sp.tau_acc) {
            if (cudaMemcpyAsync(w, p->step_tw, sizeof(float) * K, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return QST_ERR_CUDA;
            *J_out = Jt;
            *accepted = 1;
            *eta_used = eta;
            return QST_OK;
        }
    }
    *eta_used = eta / sp.eta_ratio;
    return QST_OK;
}

void qst_iter_params_default(qst_iter_params *ip) {
    if (!ip) return;
    qst_step_params_default(&ip->step);
    ip->T_alpha = 5;
    ip->T_ref = 50;
    ip->delta_window = 20;
    ip->delta_tol = 1e-4;
    ip->max_oracle_calls = 100000;
    ip->spectral = 0;
}

}  // extern "C"

namespace {
// Slot of iteration t (0 = atom, 1 = coefficients, 2 = refactor).
int iter_slot(const qst_iter_params &ip, int64_t t) {
    if (ip.T_ref > 0 && (t + 1) % ip.T_ref == 0) return 2;
    if (ip.T_alpha > 0 && (t + 1) % ip.T_alpha == 0) return 1;
    return 0;
}

qst_status graph_fail(const char *what, cudaError_t e) {
    fprintf(stderr, "qst_iterate: %s failed: %s\n", what, cudaGetErrorString(e));
    return QST_ERR_CUDA;
}
// A new condition on the graph being captured on s.  It is 0 at every launch of
// the graph until a kernel sets it.  A handle serves one conditional node.
qst_status new_condition(cudaStream_t s, cudaGraphConditionalHandle *h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusActive) return graph_fail("cudaStreamGetCaptureInfo", e);
    if ((e = cudaGraphConditionalHandleCreate(h, g, 0u, cudaGraphCondAssignDefault)) != cudaSuccess)
        return graph_fail("cudaGraphConditionalHandleCreate", e);
    return QST_OK;
}
// Conditional "if" node on the graph being captured on s, gated by `cond`;
// its body is captured on the plan's body stream, returned in *body_stream.
qst_status begin_if(qst_plan p, cudaStream_t s, cudaGraphConditionalHandle cond, cudaStream_t *body_stream) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusActive) return graph_fail("cudaStreamGetCaptureInfo", e);
    // (the parameter union has no default constructor: zeroed storage instead)
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams *np = reinterpret_cast<cudaGraphNodeParams *>(raw);
    np->type = cudaGraphNodeTypeConditional;
    np->conditional.handle = cond;
    np->conditional.type = cudaGraphCondTypeIf;
    np->conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, np)) != cudaSuccess) return graph_fail("cudaGraphAddNode", e);
    if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return graph_fail("cudaStreamUpdateCaptureDependencies", e);
    if ((e = cudaStreamBeginCaptureToGraph(p->it_body, np->conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return graph_fail("cudaStreamBeginCaptureToGraph", e);
    *body_stream = p->it_body;
    return QST_OK;
}
qst_status end_if(qst_plan p) {
    cudaGraph_t body = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->it_body, &body);
    return e == cudaSuccess ? QST_OK : graph_fail("cudaStreamEndCapture (conditional body)", e);
}

// The launch sequence of qst_iterate on stream s (captured by the caller).
// Trial j > 0 of a step grid sits in a conditional node that trial j - 1's
// acceptance kernel opens only when it rejects: once a trial is accepted the
// remaining trials are not launched at all.
qst_status iterate_sequence(qst_plan p, int T, int t0, float *psi, float *w, const uint8_t *basis,
                            const int64_t *row_ptr, const uint32_t *outcome, const uint32_t *count,
                            const uint32_t *shots, const qst_iter_params &ip, double *J_hist, int *acc_hist,
                            cudaStream_t s) {
    const qst_step_params &sp = ip.step;
    const int K = p->K;
    const int64_t D = (int64_t)1 << p->n;
    float2 *ps = reinterpret_cast<float2 *>(psi);
    float *trial = reinterpret_cast<float *>(p->step_trial);
    float *grad = reinterpret_cast<float *>(p->step_grad);
    const int *done = &p->it_state->done;
    const int *rdev = &p->it_state->r;
    // One step grid: trial j proposes (psi_t, w_t) with `propose(stream, eta)`,
    // evaluates J there and applies the acceptance rule.
    auto step_grid = [&](const float *psi_t, const float *w_t, auto &&propose) -> qst_status {
        cudaGraphConditionalHandle cur = 0, next = 0;
        double eta = sp.eta0;
        qst_status rc = QST_OK;
        for (int j = 0; j < sp.n_eta && !rc; ++j, eta *= sp.eta_ratio) {
            const int has_next = j + 1 < sp.n_eta;
            if (has_next) rc = new_condition(s, &next);
            cudaStream_t ts = s;
            bool opened = false;
            if (!rc && j > 0) {
                rc = begin_if(p, s, cur, &ts);
                opened = !rc;
            }
            if (!rc) rc = propose(ts, eta);
            if (!rc) rc = forward_core(p, psi_t, w_t, row_ptr, outcome, count, shots, nullptr, p->it_c, p->step_loss,
                                       nullptr, done, ts);
            if (!rc) rc = launch(p, QST_KERNEL_STEP, ts, [&] {
                k_iter_accept<<<1, 32, 0, ts>>>(p->it_state, p->step_loss, w_t, K, sp.mu, sp.tau_acc, j, eta, has_next,
                                                next);
            });
            if (opened) {
                const qst_status re = end_if(p);
                if (!rc) rc = re;
            }
            cur = next;
        }
        return rc;
    };
    qst_status rc = prepare(p, basis, row_ptr, outcome, shots, s);
    if (!rc) rc = forward_core(p, psi, w, row_ptr, outcome, count, shots, nullptr, p->step_c, p->step_loss, nullptr,
                               nullptr, s);
    if (!rc) rc = launch(p, QST_KERNEL_STEP, s, [&] {
        k_iter_init<<<1, 32, 0, s>>>(p->it_state, p->step_loss, w, K, sp.mu, t0 == 0 ? 1 : 0);
    });
    const int cgrid = 148 * 4;
    for (int i = 0; i < T && !rc; ++i) {
        const int slot = iter_slot(ip, (int64_t)t0 + i);
        rc = launch(p, QST_KERNEL_STEP, s, [&] { k_iter_begin<<<1, 32, 0, s>>>(p->it_state, w, K, slot); });
        if (rc) break;
        if (slot == 0) {  // atom r_t along its projected direction (Eqs. atom-direction, atom-trial)
            rc = adjoint_core(p, psi, p->step_m1, row_ptr, outcome, p->step_c, grad, nullptr, s, nullptr, done);
            if (!rc && cudaMemcpyAsync(trial, psi, sizeof(float2) * K * D, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                rc = QST_ERR_CUDA;
            if (!rc) rc = step_grid(trial, w, [&](cudaStream_t ts, double eta) {
                return launch(p, QST_KERNEL_STEP, ts, [&] {
                    k_atom_trial<<<1, 1024, 0, ts>>>(ps, p->step_grad, w, rdev, 0, eta, D, p->step_trial, done);
                });
            });
        } else if (slot == 1) {  // coefficients (Eq. coefficient-update, then P_tau)
            rc = adjoint_core(p, psi, w, row_ptr, outcome, p->step_c, grad, p->step_gw, s, nullptr, done);
            if (!rc) rc = step_grid(psi, p->step_tw, [&](cudaStream_t ts, double eta) {
                return launch(p, QST_KERNEL_STEP, ts, [&] {
                    k_coeff_trial<<<1, kProjMax, 0, ts>>>(w, p->step_gw, eta, sp.tau, K, p->step_tw, done);
                });
            });
        } else {  // exact spectral refactorisation (eta_rho = 0)
            if (cudaMemcpyAsync(trial, psi, sizeof(float2) * K * D, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(p->step_tw, w, sizeof(float) * K, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                rc = QST_ERR_CUDA;
            if (!rc) rc = qst_refactor(p, trial, p->step_tw, sp.tau, p->step_kout, s);
            if (!rc) rc = forward_core(p, trial, p->step_tw, row_ptr, outcome, count, shots, nullptr, p->it_c,
                                       p->step_loss, nullptr, nullptr, s);
            if (!rc) rc = launch(p, QST_KERNEL_STEP, s, [&] {
                k_iter_accept<<<1, 32, 0, s>>>(p->it_state, p->step_loss, p->step_tw, K, sp.mu, sp.tau_acc, 0, 0.0, 0, 0);
            });
        }
        if (!rc) rc = launch(p, QST_KERNEL_STEP, s, [&] {
            k_iter_commit<<<cgrid, 256, 0, s>>>(p->it_state, slot, p->step_trial, p->step_tw, ps, w, K, D, p->it_c,
                                                p->step_c, p->nnz);
        });
        if (!rc) rc = launch(p, QST_KERNEL_STEP, s, [&] {
            k_iter_end<<<1, 32, 0, s>>>(p->it_state, J_hist, acc_hist, i, slot, sp.n_eta, p->step_tw, K,
                                        ip.delta_window, ip.delta_tol, ip.max_oracle_calls);
        });
    }
    return rc;
}
}  // namespace

namespace {
// T iterations from t0 as one CUDA graph, captured on the first call with a
// given key and replayed afterwards (no T_rho slot runs the spectral step here).
qst_status iterate_graph(qst_plan p, int T, int t0, float *psi, float *w, const uint8_t *basis,
                         const int64_t *row_ptr, const uint32_t *outcome, const uint32_t *count,
                         const uint32_t *shots, const qst_iter_params &ip, double *J_hist, int *accepted_hist,
                         cudaStream_t st) {
    // the graph depends on the pointers, T, whether it starts a run, the slots and the parameters
    const qst_step_params &sp = ip.step;
    std::vector<double> key = {(double)(uintptr_t)psi, (double)(uintptr_t)w, (double)(uintptr_t)basis,
                               (double)(uintptr_t)row_ptr, (double)(uintptr_t)outcome, (double)(uintptr_t)count,
                               (double)(uintptr_t)shots, (double)(uintptr_t)J_hist, (double)(uintptr_t)accepted_hist,
                               (double)T, (double)(t0 == 0), sp.mu, sp.tau, sp.tau_acc, sp.eta0,
                               sp.eta_ratio, (double)sp.n_eta, (double)ip.T_alpha, (double)ip.T_ref,
                               (double)ip.delta_window, ip.delta_tol, (double)ip.max_oracle_calls};
    for (int i = 0; i < T; ++i) key.push_back((double)iter_slot(ip, (int64_t)t0 + i));
    if (!p->it_exec || key != p->it_key) {
        if (p->it_exec) {
            cudaGraphExecDestroy(p->it_exec);
            p->it_exec = nullptr;
        }
        if (!p->it_cap && cudaStreamCreateWithFlags(&p->it_cap, cudaStreamNonBlocking) != cudaSuccess)
            return QST_ERR_CUDA;
        if (!p->it_body && cudaStreamCreateWithFlags(&p->it_body, cudaStreamNonBlocking) != cudaSuccess)
            return QST_ERR_CUDA;
        const bool timing = p->timing;
        const int64_t before = p->total_launches;
        p->timing = false;  // no event records inside the graph
        if (cudaStreamBeginCapture(p->it_cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            p->timing = timing;
            return QST_ERR_CUDA;
        }
        qst_status rc = iterate_sequence(p, T, t0, psi, w, basis, row_ptr, outcome, count, shots, ip, J_hist,
                                         accepted_hist, p->it_cap);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(p->it_cap, &g);
        p->timing = timing;
        p->it_launches = p->total_launches - before;
        p->total_launches = before;
        if (rc || ce != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return rc ? rc : graph_fail("cudaStreamEndCapture", ce);
        }
        const cudaError_t ie = cudaGraphInstantiate(&p->it_exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            p->it_exec = nullptr;
            return graph_fail("cudaGraphInstantiate", ie);
        }
        p->it_key = key;
    }
    const cudaError_t le = cudaGraphLaunch(p->it_exec, st);
    if (le != cudaSuccess) return graph_fail("cudaGraphLaunch", le);
    p->total_launches += p->it_launches;
    return QST_OK;
}
}  // namespace

extern "C" {

qst_status qst_iterate(qst_plan p, int T, int t0, float *psi, float *w, const uint8_t *basis, const int64_t *row_ptr,
                       const uint32_t *outcome, const uint32_t *count, const uint32_t *shots,
                       const qst_iter_params *params, double *J_hist, int *accepted_hist, void *stream) {
    if (!p || T < 1 || t0 < 0 || !psi || !w || !basis || !row_ptr || !shots || !J_hist) return QST_ERR_INVALID_ARG;
    if (p->nnz > 0 && (!outcome || !count)) return QST_ERR_INVALID_ARG;
    if (!aligned(psi, 16) || !aligned(w, 4) || !aligned(J_hist, 8) || (accepted_hist && !aligned(accepted_hist, 4)))
        return QST_ERR_INVALID_ARG;
    qst_iter_params ip;
    qst_iter_params_default(&ip);
    if (params) ip = *params;
    const qst_step_params &sp = ip.step;
    if (sp.n_eta < 1 || !(sp.eta0 > 0.0) || !(sp.eta_ratio > 0.0) || ip.T_alpha < 0 || ip.T_ref < 0 ||
        ip.delta_window < 0 || ip.delta_window >= kIterRing || !(ip.delta_tol >= 0.0) || ip.max_oracle_calls < 0)
        return QST_ERR_INVALID_ARG;
    if (p->wide || p->K > kProjMax) return QST_ERR_UNSUPPORTED;
    if (ip.spectral != 0 && ip.spectral != 1) return QST_ERR_INVALID_ARG;
    for (int i = 0; i < T; ++i)
        if (iter_slot(ip, (int64_t)t0 + i) == 2 && !(ip.spectral ? p->lz_Q != nullptr : p->refac_C != nullptr))
            return QST_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    if (!ip.spectral) return iterate_graph(p, T, t0, psi, w, basis, row_ptr, outcome, count, shots, ip, J_hist,
                                           accepted_hist, st);
    // T_rho slots run the spectral step (qst_step slot 3, whose Krylov block sizes the host reads):
    // graph segments between them, the slot itself through qst_step, its outcome fed into the
    // device state's history and stopping rules.
    if (t0 == 0 && iter_slot(ip, 0) == 2) {  // the run starts with a T_rho slot: start the state here
        qst_status rc = prepare(p, basis, row_ptr, outcome, shots, st);
        if (!rc) rc = forward_core(p, psi, w, row_ptr, outcome, count, shots, nullptr, p->step_c, p->step_loss,
                                   nullptr, nullptr, st);
        if (!rc) rc = launch(p, QST_KERNEL_STEP, st, [&] {
            k_iter_init<<<1, 32, 0, st>>>(p->it_state, p->step_loss, w, p->K, sp.mu, 1);
        });
        if (rc) return rc;
    }
    // segments write their history into plan-owned buffers, so every segment with the same
    // slots replays one graph; the history is then copied into place
    int seg_max = 0;
    for (int i = 0, len = 0; i < T; ++i) {
        len = iter_slot(ip, (int64_t)t0 + i) == 2 ? 0 : len + 1;
        seg_max = len > seg_max ? len : seg_max;
    }
    if (seg_max > p->it_seg_cap) {
        cudaFree(p->it_Jseg);
        cudaFree(p->it_aseg);
        p->it_Jseg = nullptr;
        p->it_aseg = nullptr;
        p->it_seg_cap = 0;
        if (cudaMalloc(&p->it_Jseg, sizeof(double) * seg_max) != cudaSuccess ||
            cudaMalloc(&p->it_aseg, sizeof(int) * seg_max) != cudaSuccess) {
            cudaGetLastError();
            return QST_ERR_NO_MEMORY;
        }
        p->it_seg_cap = seg_max;
    }
    for (int i = 0; i < T;) {
        int j = i;
        while (j < T && iter_slot(ip, (int64_t)t0 + j) != 2) ++j;
        if (j > i) {
            qst_status rc = iterate_graph(p, j - i, t0 + i, psi, w, basis, row_ptr, outcome, count, shots, ip,
                                          p->it_Jseg, p->it_aseg, st);
            if (!rc && (cudaMemcpyAsync(J_hist + i, p->it_Jseg, sizeof(double) * (j - i), cudaMemcpyDeviceToDevice,
                                        st) != cudaSuccess ||
                        (accepted_hist && cudaMemcpyAsync(accepted_hist + i, p->it_aseg, sizeof(int) * (j - i),
                                                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)))
                rc = QST_ERR_CUDA;
            if (rc) return rc;
        }
        if (j == T) break;
        int stopped = 0;
        if (cudaMemcpyAsync(&stopped, &p->it_state->stopped, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return QST_ERR_CUDA;
        double J = 0.0, eta = 0.0;
        int acc = 0;
        long long calls = 0;
        if (!stopped) {
            const qst_status rc = qst_step(p, 3, 0, psi, w, basis, row_ptr, outcome, count, shots, &ip.step, &J, &acc,
                                           &eta, stream);
            if (rc) return rc;
            calls = p->step_calls;
        }
        const qst_status rc = launch(p, QST_KERNEL_STEP, st, [&] {
            k_iter_external<<<1, 32, 0, st>>>(p->it_state, J_hist, accepted_hist, j, J, acc, calls, ip.delta_window,
                                              ip.delta_tol, ip.max_oracle_calls);
        });
        if (rc) return rc;
        i = j + 1;
    }
    return QST_OK;
}

qst_status qst_iterate_state(qst_plan p, int *stopped, long long *oracle_calls, int *accepted_updates,
                             double *J) {
    if (!p || !p->it_state) return QST_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return QST_ERR_CUDA;
    IterState h;
    if (cudaMemcpy(&h, p->it_state, sizeof(IterState), cudaMemcpyDeviceToHost) != cudaSuccess) return QST_ERR_CUDA;
    if (stopped) *stopped = h.stopped;
    if (oracle_calls) *oracle_calls = h.oracle_calls;
    if (accepted_updates) *accepted_updates = h.n_acc;
    if (J) *J = h.J;
    return QST_OK;
}

qst_status qst_refactor(qst_plan p, float *psi, float *w, double tau, int *K_out, void *stream) {
    if (!p || !psi || !w || !K_out) return QST_ERR_INVALID_ARG;
    if (p->K > kRefacMax || !p->refac_C) return QST_ERR_UNSUPPORTED;
    if (!aligned(psi, 16) || !aligned(w, 4) || !aligned(K_out, 4)) return QST_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int K = p->K;
    const int64_t D = (int64_t)1 << p->n;
    float2 *ps = reinterpret_cast<float2 *>(psi);
    qst_status rc = launch(p, QST_KERNEL_REFACTOR, st, [&] {
        k_gram<<<K * (K + 1) / 2, 256, 0, st>>>(ps, K, D, p->refac_C);
    });
    if (rc) return rc;
    rc = launch(p, QST_KERNEL_REFACTOR, st, [&] {
        k_eig<<<1, kRefacMax, 0, st>>>(p->refac_C, w, K, tau, p->refac_T, w, K_out);
    });
    if (rc) return rc;
    const int64_t blocks = (D + 255) / 256;
    const int grid = (int)(blocks < 148 * 8 ? blocks : 148 * 8);
    return launch(p, QST_KERNEL_REFACTOR, st, [&] { k_combine<<<grid, 256, 0, st>>>(ps, K, D, p->refac_T); });
}

}  // extern "C"

// ----------------------------------------------------------------- adjoint without allocation
//
// qst_adjoint_noalloc serves callers that cannot call cudaMalloc: code running
// under an allocator it does not own (a framework's caching pool, a sandbox
// that forbids raw device allocation), or loops that must not trigger
// cudaMalloc's implicit device synchronisation.  Its workspace is this
// file-scope device array instead of a plan's cudaMalloc'd buffers.  Every GPU
// that loads the library holds the array until the process exits.

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[QST_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The first call
// on a device looks it up (cudaGetSymbolAddress, with that device current) and
// sets the kernels' shared-memory limits; later calls reuse the address.
qst_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return QST_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return QST_ERR_CUDA;
        }
        for (int c = 1; c <= kMaxChunk; ++c)
            for (int ra = 4; ra <= 5; ++ra)
                with_geo(c, ra, [](auto cc, auto rr) { set_smem_attrs<decltype(cc)::value, decltype(rr)::value>(); });
        if (cudaGetLastError() != cudaSuccess) return QST_ERR_CUDA;
        g_noalloc_ptr[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    return QST_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" qst_status qst_adjoint_noalloc(int n, int M, int K, int64_t nnz, const qst_params *params,
                                          const float *psi, const float *w, const uint8_t *basis,
                                          const int64_t *row_ptr, const uint32_t *outcome, const float *c_obs,
                                          float *grad_psi, float *grad_w, int *device_status, void *stream) {
    if (n < 1 || M < 1 || K < 1 || nnz < 0 || !device_status) return QST_ERR_INVALID_ARG;
    if (nnz > (int64_t)M << n) return QST_ERR_INVALID_ARG;
    qst_params prm;
    qst_params_default(&prm);
    if (params) prm = *params;
    if (!(prm.eps >= 0.0) || prm.norm_settings < 0 || prm.max_bin_settings < 0) return QST_ERR_INVALID_ARG;
    // always the per-setting-round kernels: a request for another family is refused
    if (prm.fixed_rounds != -1 && prm.fixed_rounds != 0) return QST_ERR_INVALID_ARG;
    if (prm.precision != 0) return QST_ERR_UNSUPPORTED;  // the FP32 per-setting-round kernels only
    const int c = prm.chunk_qubits ? prm.chunk_qubits : (n < kMaxChunk ? n : kMaxChunk);
    if (c < 1 || c > kMaxChunk || c > n) return QST_ERR_INVALID_ARG;
    const int r = n - c;
    if (r > kMaxTop || K > 4096 || M > (1 << 24) || nnz > ((int64_t)1 << 31) - 1) return QST_ERR_UNSUPPORTED;
    const int ra = prm.reg_bits ? prm.reg_bits : kDefaultRegBits;
    if (ra != 4 && ra != 5) return QST_ERR_INVALID_ARG;
    // Fewest bins (largest bins) keep the z buffer small.
    const int smax = prm.max_bin_settings ? (prm.max_bin_settings < kMaxBin ? prm.max_bin_settings : kMaxBin)
                                          : kMaxBin;
    const int nkeys = ipow3(r);
    const int nb_max = (nkeys < M ? nkeys : M) + (M + smax - 1) / smax;
    const size_t D = (size_t)1 << n;
    // scratch layout
    size_t off = 0;
    const size_t o_nbins = off; off += align256(sizeof(int));
    const size_t o_bins = off; off += align256((size_t)nb_max * sizeof(Bin));
    const size_t o_plans = off; off += align256((size_t)M * sizeof(SetPlan));
    const size_t o_order = off; off += align256((size_t)M * sizeof(int32_t));
    const size_t o_choff = off; off += align256((size_t)M * ((1u << r) + 1) * sizeof(int32_t));
    const size_t o_hdot = off; off += align256(((size_t)K << c) * sizeof(double));
    const size_t o_zbuf = off; off += align256((size_t)nb_max * K * D * sizeof(float2));
    if (off > (size_t)QST_NOALLOC_SCRATCH_BYTES) {
        fprintf(stderr, "qst_adjoint_noalloc: needs %zu bytes of workspace, the scratch holds %u\n", off,
                (unsigned)QST_NOALLOC_SCRATCH_BYTES);
        return QST_ERR_SCRATCH_TOO_SMALL;
    }
    unsigned char *base = nullptr;
    qst_status rc = noalloc_scratch(&base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // The device status word is the caller's; it must start at zero.
    if (cudaMemsetAsync(device_status, 0, sizeof(int), st) != cudaSuccess) return QST_ERR_CUDA;
    // A plan object on the stack whose workspace pointers point into the
    // scratch; qst_adjoint then runs unchanged and allocates nothing.
    qst_plan_s tmp;
    tmp.n = n;
    tmp.M = M;
    tmp.K = K;
    tmp.nnz = nnz;
    tmp.prm = prm;
    tmp.c = c;
    tmp.r = r;
    tmp.A = c < ra ? c : ra;
    tmp.T = 1 << (c - tmp.A);
    tmp.B = prm.norm_settings ? prm.norm_settings : M;
    tmp.smax = smax;
    tmp.nb_max = nb_max;
    cudaGetDevice(&tmp.device);
    tmp.n_bins = reinterpret_cast<int *>(base + o_nbins);
    tmp.bins = reinterpret_cast<Bin *>(base + o_bins);
    tmp.plans = reinterpret_cast<SetPlan *>(base + o_plans);
    tmp.order = reinterpret_cast<int32_t *>(base + o_order);
    tmp.choff = reinterpret_cast<int32_t *>(base + o_choff);
    tmp.hdot = reinterpret_cast<double *>(base + o_hdot);
    tmp.zbuf = reinterpret_cast<float2 *>(base + o_zbuf);
    tmp.status = device_status;
    // tmp owns nothing: its workspace pointers are views of the scratch array
    return qst_adjoint(&tmp, psi, w, basis, row_ptr, outcome, c_obs, grad_psi, grad_w, stream);
}

// ----------------------------------------------------------------- batched instances
//
// Many independent instances of uneven shape (n, M, K, nnz): one plan per
// instance, and one CUDA graph per set of buffers.  The graph forks every
// instance's forward + adjoint onto its own stream, so the instances run
// concurrently and the whole batch is one graph launch.

namespace {

// Argument records of qst_batch_evaluate's multi-instance launches (one per
// instance and launch; the unit kernels take FwdArgs / AdjArgs).
struct PackArgs {
    const uint8_t *basis;
    int M, n, c, r, smax, areg;
    SetPlan *plans;
    int32_t *order;
    Bin *bins;
    int *n_bins, *status;
};
struct ValArgs {
    const int64_t *row_ptr;
    const uint32_t *outcome, *shots;
    int M;
    int64_t nnz;
    int n, c, r, validate;
    int32_t *choff;
    int *status;
};
struct EpiArgs {
    const float *ppart;
    const int64_t *row_ptr;
    const uint32_t *count, *shots;
    int M, K;
    int64_t nnz;
    float invB, eps;
    float *c_obs;
    double *loss_part;
};
struct LossArgs {
    const double *loss_part;
    int parts;
    double *loss;
    int *status;
};
struct RedArgs {
    const float2 *zbuf;
    const Bin *bins;
    const int *n_bins;
    const float *w;
    const float2 *psi;
    float2 *grad;
    double *hdot;
    int n, c, K, r;
    float invB;
};
struct HsumArgs {
    const double *hdot;
    int c;
    float invB;
    float *grad_w;
};

__global__ void __launch_bounds__(1024) k_pack_multi(const PackArgs *__restrict__ args) {
    const PackArgs a = args[blockIdx.x];
    pack_body(a.basis, a.M, a.n, a.c, a.r, a.smax, a.areg, a.plans, a.order, a.bins, a.n_bins, a.status, 0);
}
__global__ void __launch_bounds__(256) k_validate_multi(const ValArgs *__restrict__ args, const int *__restrict__ start,
                                                        int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const ValArgs a = args[i];
    validate_body(a.row_ptr, a.outcome, a.shots, a.M, a.nnz, a.n, a.c, a.r, a.validate, a.choff, a.status,
                  (int)blockIdx.x - start[i]);
}
__global__ void __launch_bounds__(256) k_fwd_epilogue_multi(const EpiArgs *__restrict__ args,
                                                            const int *__restrict__ start, int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const EpiArgs a = args[i];
    epilogue_body<true>(a.ppart, a.row_ptr, a.count, a.shots, a.M, a.K, a.nnz, a.invB, a.eps, nullptr, a.c_obs,
                  a.loss_part, nullptr, (int)blockIdx.x - start[i]);
}
__global__ void __launch_bounds__(256) k_loss_multi(const LossArgs *__restrict__ args) {
    const LossArgs a = args[blockIdx.x];
    loss_body(a.loss_part, a.parts, a.loss, a.status, nullptr, 0);
}
__global__ void __launch_bounds__(256) k_reduce_multi(const RedArgs *__restrict__ args, const int *__restrict__ start,
                                                      int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const RedArgs a = args[i];
    const int cta = (int)blockIdx.x - start[i];
    switch (a.r) {
        case 0: reduce_body<0>(a.zbuf, a.bins, a.n_bins, a.w, a.psi, a.grad, a.hdot, a.n, a.c, a.K, a.invB, nullptr, cta); break;
        case 1: reduce_body<1>(a.zbuf, a.bins, a.n_bins, a.w, a.psi, a.grad, a.hdot, a.n, a.c, a.K, a.invB, nullptr, cta); break;
        case 2: reduce_body<2>(a.zbuf, a.bins, a.n_bins, a.w, a.psi, a.grad, a.hdot, a.n, a.c, a.K, a.invB, nullptr, cta); break;
        case 3: reduce_body<3>(a.zbuf, a.bins, a.n_bins, a.w, a.psi, a.grad, a.hdot, a.n, a.c, a.K, a.invB, nullptr, cta); break;
        default: reduce_body<4>(a.zbuf, a.bins, a.n_bins, a.w, a.psi, a.grad, a.hdot, a.n, a.c, a.K, a.invB, nullptr, cta); break;
    }
}
__global__ void __launch_bounds__(256) k_hsum_multi(const HsumArgs *__restrict__ args, const int *__restrict__ start,
                                                    int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const HsumArgs a = args[i];
    hsum_body(a.hdot, a.c, a.invB, a.grad_w, nullptr, (int)blockIdx.x - start[i]);
}

// Chunk-kernel family of a plan: the multi-instance forward / adjoint
// launches group instances by it (same kernel, block and shared memory).
// >= 0: generic kernels, 100 c + A; -10 - n: warp-unit kernels of n qubits
enum { kFam2rCache = -1, kFam2r = -2, kFamFx = -3, kFam2rCache11 = -4, kFam2rCache10 = -5, kFam2r11 = -6, kFam2r10 = -7 };
int plan_family(const qst_plan_s *p) {
    if (p->fw) return -10 - p->n;
    if (p->fx2 && p->c == 11) return p->cache_on ? kFam2rCache11 : kFam2r11;
    if (p->fx2 && p->c == 10) return p->cache_on ? kFam2rCache10 : kFam2r10;
    if (p->fx2) return p->cache_on ? kFam2rCache : kFam2r;
    if (p->fx) return kFamFx;
    return 100 * p->c + p->A;
}
// CTAs of one instance's forward / adjoint grid
int64_t plan_unit_ctas(const qst_plan_s *p) {
    const int64_t units = (int64_t)p->nb_max << p->r;
    if (p->fw) return (units * p->K + kWuT / 32 - 1) / (kWuT / 32);
    return units * (p->fx2 ? k2_atom_groups(p->K, p->c) : p->K);
}

constexpr int kBatchStreams = 16;
constexpr int kBatchBin = 64;  // settings per bin of a batch plan of 10..16 qubits (see batch_create)

enum BatchPhase { kPhPack, kPhValidate, kPhForward, kPhEpilogue, kPhLoss, kPhAdjoint, kPhReduce, kPhHsum, kPhases };

// One multi-instance launch: its grid, and where its argument records and
// CTA starts sit in the batch's device argument buffer.
struct BatchLaunch {
    int phase, family;
    int grid, count;
    size_t args_off, start_off;
};

}  // namespace

struct qst_batch_s {
    int count = 0;
    std::vector<qst_plan> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> fork, join;
    cudaEvent_t start = nullptr;
    cudaStream_t cap = nullptr;  // capture stream (the caller's may be the legacy default stream)
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> key;  // buffers the graph was captured with
    bool multi = false;             // every plan has a multi-instance kernel family
    cudaGraphExec_t it_exec = nullptr;  // qst_batch_iterate's graph and its key
    std::vector<double> it_key;
    unsigned char *dev_args = nullptr;
    size_t dev_bytes = 0;
    std::vector<BatchLaunch> launches;
};

extern "C" qst_status qst_batch_destroy(qst_batch b) {
    if (!b) return QST_ERR_INVALID_ARG;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->it_exec) cudaGraphExecDestroy(b->it_exec);
    for (auto p : b->plans)
        if (p) qst_plan_destroy(p);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto e : b->fork) cudaEventDestroy(e);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->start) cudaEventDestroy(b->start);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->dev_args);
    delete b;
    return QST_OK;
}

namespace {
// Dynamic shared memory limits of the multi-instance chunk kernels of a family.
void set_family_attrs(int fam) {
    if (fam == kFam2rCache || fam == kFam2r) {
        cudaFuncSetAttribute(k_forward_2r_multi<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
        cudaFuncSetAttribute(k_forward_2r_multi<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
        cudaFuncSetAttribute(k_adjoint_2c_multi<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2c_smem(k2cStageMulti).total);
        cudaFuncSetAttribute(k_adjoint_2r_multi<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2p_smem().total);
    } else if (fam == kFam2rCache11) {
        cudaFuncSetAttribute(k_forward_2r_multi<true, 11>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
        cudaFuncSetAttribute(k_adjoint_2c_multi<11>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2c_smem(k2cStageMulti).total);
    } else if (fam == kFam2rCache10) {
        cudaFuncSetAttribute(k_forward_2r_multi<true, 10>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
        cudaFuncSetAttribute(k_adjoint_2c_multi<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2c_smem(k2cStageMulti).total);
    } else if (fam == kFam2r11) {
        cudaFuncSetAttribute(k_forward_2r_multi<false, 11>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
        cudaFuncSetAttribute(k_adjoint_2r_multi<11>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2p_smem().total);
    } else if (fam == kFam2r10) {
        cudaFuncSetAttribute(k_forward_2r_multi<false, 10>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_smem_fwd().total);
        cudaFuncSetAttribute(k_adjoint_2r_multi<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2p_smem().total);
    } else if (fam <= -15) {
        // at most 16 KB of shared memory: no attribute
    } else if (fam == kFamFx) {
        cudaFuncSetAttribute(k_forward_fx_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, fx_smem(false).total);
        cudaFuncSetAttribute(k_adjoint_fx_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, fx_smem(true).total);
    } else {
        with_geo(fam / 100, fam % 100, [](auto cc, auto ra) {
            constexpr int C = decltype(cc)::value, RA = decltype(ra)::value;
            cudaFuncSetAttribute(k_forward_multi<C, RA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_plan(C, false).total);
            cudaFuncSetAttribute(k_adjoint_multi<C, RA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_plan(C, true).total);
        });
    }
}
}  // namespace

namespace {
// params: one record for all instances (each == false; the batch bin rule
// below applies) or one per instance (each == true; taken as given).
qst_status batch_create(qst_batch *out, int count, const int *n, const int *M, const int *K, const int64_t *nnz,
                        const qst_params *params, bool each) {
    if (!out || count < 1 || !n || !M || !K || !nnz || (each && !params)) return QST_ERR_INVALID_ARG;
    *out = nullptr;
    qst_batch b = new (std::nothrow) qst_batch_s;
    if (!b) return QST_ERR_NO_MEMORY;
    b->count = count;
    b->plans.assign(count, nullptr);
    // The instances share the GPU, so a plan of 10..16 qubits needs no small bins
    // to fill it alone: unless the caller fixes max_bin_settings, such plans bin
    // up to kBatchBin settings (12-qubit chunks then run the two-round kernels).
    // On the 64-instance workload bins of 64 measured 15.08 ms per evaluation,
    // 32 15.54 and 96 15.17 (for the 12..14- and the 10, 11-qubit classes
    // alike).  Smaller states keep their own bin sizes: their units are a warp
    // per (bin, atom), and many short bins keep the SMs busy.
    qst_params prm0;
    qst_params_default(&prm0);
    if (params && !each) prm0 = *params;
    for (int i = 0; i < count; ++i) {
        qst_params prm = each ? params[i] : prm0;
        if (!each && prm0.max_bin_settings == 0 && n[i] >= 10 && n[i] <= kMaxChunk + kMaxTop)
            prm.max_bin_settings = kBatchBin;
        const qst_status rc = qst_plan_create(&b->plans[i], n[i], M[i], K[i], nnz[i], &prm);
        if (rc) {
            qst_batch_destroy(b);
            return rc;
        }
    }
    // multi-instance launches for every plan off the wide path and off the tensor cores
    b->multi = true;
    for (auto p : b->plans)
        if (p->wide || p->cl || p->prm.precision > 0) b->multi = false;
    if (b->multi) {
        for (auto p : b->plans) set_family_attrs(plan_family(p));
        if (cudaGetLastError() != cudaSuccess) {
            qst_batch_destroy(b);
            return QST_ERR_CUDA;
        }
    }
    const int ns = count < kBatchStreams ? count : kBatchStreams;
    b->streams.assign(ns, nullptr);
    b->fork.assign(ns, nullptr);
    b->join.assign(ns, nullptr);
    bool ok = cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
    for (int j = 0; j < ns && ok; ++j)
        ok = cudaStreamCreateWithFlags(&b->streams[j], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->fork[j], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        qst_batch_destroy(b);
        return QST_ERR_CUDA;
    }
    *out = b;
    return QST_OK;
}
}  // namespace

extern "C" qst_status qst_batch_create(qst_batch *out, int count, const int *n, const int *M, const int *K,
                                       const int64_t *nnz, const qst_params *params) {
    return batch_create(out, count, n, M, K, nnz, params, false);
}

extern "C" qst_status qst_batch_create_each(qst_batch *out, int count, const int *n, const int *M, const int *K,
                                            const int64_t *nnz, const qst_params *params) {
    return batch_create(out, count, n, M, K, nnz, params, true);
}

extern "C" qst_status qst_batch_plan(qst_batch b, int i, qst_plan *plan) {
    if (!b || !plan || i < 0 || i >= b->count) return QST_ERR_INVALID_ARG;
    *plan = b->plans[i];
    return QST_OK;
}

namespace {
// Host-side image of the device argument buffer (16-byte aligned arrays).
struct ArgImage {
    std::vector<unsigned char> bytes;
    template <typename T>
    size_t put(const std::vector<T> &v) {
        const size_t off = (bytes.size() + 15) & ~(size_t)15;
        bytes.resize(off + v.size() * sizeof(T));
        if (!v.empty()) memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

// Argument records and launches of one batch evaluation.  Per phase, one
// launch per kernel family; within a family the instances with the most
// settings per bin come first, so their long CTAs start first.
qst_status batch_build(qst_batch b, const float *const *psi, const float *const *w, const uint8_t *const *basis,
                       const int64_t *const *row_ptr, const uint32_t *const *outcome, const uint32_t *const *count,
                       const uint32_t *const *shots, double *const *loss, float *const *c_obs,
                       float *const *grad_psi, float *const *grad_w) {
    ArgImage img;
    b->launches.clear();
    const int N = b->count;
    auto add = [&](int phase, int family, const std::vector<int> &grid_of, size_t args_off) {
        std::vector<int> start(grid_of.size() + 1, 0);
        for (size_t i = 0; i < grid_of.size(); ++i) start[i + 1] = start[i] + grid_of[i];
        BatchLaunch L;
        L.phase = phase;
        L.family = family;
        L.grid = start.back();
        L.count = (int)grid_of.size();
        L.args_off = args_off;
        L.start_off = img.put(start);
        if (L.grid > 0) b->launches.push_back(L);
    };
    {
        std::vector<PackArgs> a(N);
        std::vector<int> g(N, 1);
        for (int i = 0; i < N; ++i) {
            const qst_plan p = b->plans[i];
            a[i] = PackArgs{basis[i], p->M, p->n, p->c, p->r, p->smax, p->A, p->plans, p->order, p->bins,
                            p->n_bins, p->status};
        }
        add(kPhPack, 0, g, img.put(a));
    }
    {
        std::vector<ValArgs> a(N);
        std::vector<int> g(N);
        for (int i = 0; i < N; ++i) {
            const qst_plan p = b->plans[i];
            a[i] = ValArgs{row_ptr[i], outcome[i], shots[i], p->M, p->nnz, p->n, p->c, p->r, p->prm.validate,
                           p->choff, p->status};
            g[i] = (p->M + 7) / 8;
        }
        add(kPhValidate, 0, g, img.put(a));
    }
    // kernel families, instances ordered by settings per bin (descending)
    std::vector<int> fams;
    for (auto p : b->plans) {
        const int f = plan_family(p);
        if (std::find(fams.begin(), fams.end(), f) == fams.end()) fams.push_back(f);
    }
    std::vector<std::vector<int>> members(fams.size());
    for (size_t fi = 0; fi < fams.size(); ++fi) {
        for (int i = 0; i < N; ++i)
            if (plan_family(b->plans[i]) == fams[fi]) members[fi].push_back(i);
        std::stable_sort(members[fi].begin(), members[fi].end(),
                         [&](int x, int y) { return b->plans[x]->smax > b->plans[y]->smax; });
    }
    for (size_t fi = 0; fi < fams.size(); ++fi) {
        std::vector<FwdArgs> a;
        std::vector<int> g;
        for (int i : members[fi]) {
            const qst_plan p = b->plans[i];
            FwdArgs f;
            f.psi = reinterpret_cast<const float2 *>(psi[i]);
            f.w = w[i];
            f.plans = p->plans;
            f.order = p->order;
            f.bins = p->bins;
            f.n_bins = p->n_bins;
            f.row_ptr = row_ptr[i];
            f.outcome = outcome[i];
            f.choff = p->choff;
            f.ppart = p->ppart;
            f.p_dense = nullptr;
            f.nnz = p->nnz;
            f.src_bin_stride = 0;
            f.skip = nullptr;
            f.n = p->n;
            f.r = p->r;
            f.K = p->K;
            f.phi_obs = p->cache_on ? p->phi : nullptr;
            f.tc_ops = p->tc_ops;
            f.status = p->status;
            a.push_back(f);
            g.push_back((int)plan_unit_ctas(p));
        }
        add(kPhForward, fams[fi], g, img.put(a));
    }
    {
        std::vector<EpiArgs> a(N);
        std::vector<LossArgs> la(N);
        std::vector<int> g(N), one(N, 1);
        for (int i = 0; i < N; ++i) {
            const qst_plan p = b->plans[i];
            a[i] = EpiArgs{p->ppart, row_ptr[i], count[i], shots[i], p->M, p->K, p->nnz, 1.0f / (float)p->B,
                           (float)p->prm.eps, c_obs[i], p->loss_part};
            g[i] = p->loss_parts;
            la[i] = LossArgs{p->loss_part, p->loss_parts, loss[i], p->status};
        }
        add(kPhEpilogue, 0, g, img.put(a));
        add(kPhLoss, 0, one, img.put(la));
    }
    for (size_t fi = 0; fi < fams.size(); ++fi) {
        std::vector<AdjArgs> a;
        std::vector<int> g;
        for (int i : members[fi]) {
            const qst_plan p = b->plans[i];
            AdjArgs d;
            d.psi = reinterpret_cast<const float2 *>(psi[i]);
            d.plans = p->plans;
            d.order = p->order;
            d.bins = p->bins;
            d.n_bins = p->n_bins;
            d.row_ptr = row_ptr[i];
            d.outcome = outcome[i];
            d.c_obs = c_obs[i];
            d.choff = p->choff;
            d.zbuf = p->zbuf;
            d.src_bin_stride = 0;
            d.n = p->n;
            d.r = p->r;
            d.K = p->K;
            d.phi_obs = p->cache_on ? p->phi : nullptr;
            d.nnz = p->nnz;
            d.skip = nullptr;
            d.tc_ops = p->tc_ops;
            d.status = p->status;
            a.push_back(d);
            g.push_back((int)plan_unit_ctas(p));
        }
        add(kPhAdjoint, fams[fi], g, img.put(a));
    }
    {
        std::vector<RedArgs> a(N);
        std::vector<HsumArgs> h(N);
        std::vector<int> g(N), gk(N);
        for (int i = 0; i < N; ++i) {
            const qst_plan p = b->plans[i];
            const float invB = 1.0f / (float)p->B;
            a[i] = RedArgs{p->zbuf, p->bins, p->n_bins, w[i], reinterpret_cast<const float2 *>(psi[i]),
                           reinterpret_cast<float2 *>(grad_psi[i]), p->hdot, p->n, p->c, p->K, p->r, invB};
            g[i] = (int)((((int64_t)p->K << p->c) + 255) / 256);
            h[i] = HsumArgs{p->hdot, p->c, invB, grad_w[i]};
            gk[i] = p->K;
        }
        add(kPhReduce, 0, g, img.put(a));
        add(kPhHsum, 0, gk, img.put(h));
    }
    if (img.bytes.size() > b->dev_bytes) {
        cudaFree(b->dev_args);
        b->dev_args = nullptr;
        b->dev_bytes = 0;
        if (cudaMalloc(&b->dev_args, img.bytes.size()) != cudaSuccess) {
            cudaGetLastError();
            return QST_ERR_NO_MEMORY;
        }
        b->dev_bytes = img.bytes.size();
    }
    if (cudaMemcpy(b->dev_args, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return QST_ERR_CUDA;
    return QST_OK;
}

void batch_launch(qst_batch b, const BatchLaunch &L, cudaStream_t st) {
    const unsigned char *base = b->dev_args;
    const int *start = reinterpret_cast<const int *>(base + L.start_off);
    const void *args = base + L.args_off;
    const int grid = L.grid, cnt = L.count, fam = L.family;
    switch (L.phase) {
        case kPhPack: k_pack_multi<<<grid, 1024, 0, st>>>(static_cast<const PackArgs *>(args)); break;
        case kPhValidate:
            k_validate_multi<<<grid, 256, 0, st>>>(static_cast<const ValArgs *>(args), start, cnt);
            break;
        case kPhEpilogue:
            k_fwd_epilogue_multi<<<grid, 256, 0, st>>>(static_cast<const EpiArgs *>(args), start, cnt);
            break;
        case kPhLoss: k_loss_multi<<<grid, 256, 0, st>>>(static_cast<const LossArgs *>(args)); break;
        case kPhReduce: k_reduce_multi<<<grid, 256, 0, st>>>(static_cast<const RedArgs *>(args), start, cnt); break;
        case kPhHsum: k_hsum_multi<<<grid, 256, 0, st>>>(static_cast<const HsumArgs *>(args), start, cnt); break;
        case kPhForward: {
            const FwdArgs *a = static_cast<const FwdArgs *>(args);
            if (fam == kFam2rCache) k_forward_2r_multi<true><<<grid, k2T, k2_smem_fwd().total, st>>>(a, start, cnt);
            else if (fam == kFam2r) k_forward_2r_multi<false><<<grid, k2T, k2_smem_fwd().total, st>>>(a, start, cnt);
            else if (fam == kFam2rCache11) k_forward_2r_multi<true, 11><<<grid, k2T, k2_smem_fwd().total, st>>>(a, start, cnt);
            else if (fam == kFam2rCache10) k_forward_2r_multi<true, 10><<<grid, k2T, k2_smem_fwd().total, st>>>(a, start, cnt);
            else if (fam == kFam2r11) k_forward_2r_multi<false, 11><<<grid, k2T, k2_smem_fwd().total, st>>>(a, start, cnt);
            else if (fam == kFam2r10) k_forward_2r_multi<false, 10><<<grid, k2T, k2_smem_fwd().total, st>>>(a, start, cnt);
            else if (fam == kFamFx) k_forward_fx_multi<<<grid, kFxT, fx_smem(false).total, st>>>(a, start, cnt);
            else if (fam <= -15)
                with_wu(-10 - fam, [&](auto nb) {
                    constexpr int NB = decltype(nb)::value;
                    k_forward_wu_multi<NB><<<grid, kWuT, wu_smem(NB), st>>>(a, start, cnt);
                });
            else
                with_geo(fam / 100, fam % 100, [&](auto cc, auto ra) {
                    constexpr int C = decltype(cc)::value, RA = decltype(ra)::value;
                    k_forward_multi<C, RA><<<grid, Geo<C, RA>::T, smem_plan(C, false).total, st>>>(a, start, cnt);
                });
            break;
        }
        case kPhAdjoint: {
            const AdjArgs *a = static_cast<const AdjArgs *>(args);
            if (fam == kFam2rCache) k_adjoint_2c_multi<12><<<grid, k2T, k2c_smem(k2cStageMulti).total, st>>>(a, start, cnt);
            else if (fam == kFam2rCache11) k_adjoint_2c_multi<11><<<grid, k2T, k2c_smem(k2cStageMulti).total, st>>>(a, start, cnt);
            else if (fam == kFam2rCache10) k_adjoint_2c_multi<10><<<grid, k2T, k2c_smem(k2cStageMulti).total, st>>>(a, start, cnt);
            else if (fam == kFam2r) k_adjoint_2r_multi<12><<<grid, k2T, k2p_smem().total, st>>>(a, start, cnt);
            else if (fam == kFam2r11) k_adjoint_2r_multi<11><<<grid, k2T, k2p_smem().total, st>>>(a, start, cnt);
            else if (fam == kFam2r10) k_adjoint_2r_multi<10><<<grid, k2T, k2p_smem().total, st>>>(a, start, cnt);
            else if (fam == kFamFx) k_adjoint_fx_multi<<<grid, kFxT, fx_smem(true).total, st>>>(a, start, cnt);
            else if (fam <= -15)
                with_wu(-10 - fam, [&](auto nb) {
                    constexpr int NB = decltype(nb)::value;
                    k_adjoint_wu_multi<NB><<<grid, kWuT, wu_smem(NB), st>>>(a, start, cnt);
                });
            else
                with_geo(fam / 100, fam % 100, [&](auto cc, auto ra) {
                    constexpr int C = decltype(cc)::value, RA = decltype(ra)::value;
                    k_adjoint_multi<C, RA><<<grid, Geo<C, RA>::T, smem_plan(C, true).total, st>>>(a, start, cnt);
                });
            break;
        }
        default: break;
    }
}
}  // namespace

extern "C" qst_status qst_batch_evaluate(qst_batch b, const float *const *psi, const float *const *w,
                                         const uint8_t *const *basis, const int64_t *const *row_ptr,
                                         const uint32_t *const *outcome, const uint32_t *const *count,
                                         const uint32_t *const *shots, double *const *loss, float *const *c_obs,
                                         float *const *grad_psi, float *const *grad_w, void *stream) {
    if (!b || !psi || !w || !basis || !row_ptr || !outcome || !count || !shots || !loss || !c_obs || !grad_psi ||
        !grad_w)
        return QST_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<const void *> key;
    key.reserve((size_t)b->count * 11);
    for (int i = 0; i < b->count; ++i) {
        const void *ptrs[11] = {psi[i], w[i], basis[i], row_ptr[i], outcome[i], count[i], shots[i],
                                loss[i], c_obs[i], grad_psi[i], grad_w[i]};
        for (const void *q : ptrs) key.push_back(q);
        if (!psi[i] || !w[i] || !basis[i] || !row_ptr[i] || !shots[i] || !loss[i] || !grad_psi[i] || !grad_w[i])
            return QST_ERR_INVALID_ARG;
    }
    if (!b->exec || key != b->key) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        if (b->multi) {
            const qst_status rb = batch_build(b, psi, w, basis, row_ptr, outcome, count, shots, loss, c_obs, grad_psi,
                                              grad_w);
            if (rb) return rb;
        }
        cudaGraph_t graph = nullptr;
        cudaStream_t cs = b->cap;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return QST_ERR_CUDA;
        }
        qst_status rc = QST_OK;
        const int ns = (int)b->streams.size();
        if (!b->multi) {
            if (cudaEventRecord(b->start, cs) != cudaSuccess) rc = QST_ERR_CUDA;
            for (int j = 0; j < ns && !rc; ++j)
                if (cudaStreamWaitEvent(b->streams[j], b->start, 0) != cudaSuccess) rc = QST_ERR_CUDA;
        }
        if (b->multi) {
            // one launch per phase and kernel family; a phase's families run on forked streams
            for (int ph = 0; ph < kPhases && !rc; ++ph) {
                std::vector<const BatchLaunch *> L;
                for (const auto &l : b->launches)
                    if (l.phase == ph) L.push_back(&l);
                if (L.size() == 1) {
                    batch_launch(b, *L[0], cs);
                    continue;
                }
                if (L.empty()) continue;
                if (cudaEventRecord(b->start, cs) != cudaSuccess) rc = QST_ERR_CUDA;
                const int used = (int)L.size() < ns ? (int)L.size() : ns;
                for (int j = 0; j < used && !rc; ++j)
                    if (cudaStreamWaitEvent(b->streams[j], b->start, 0) != cudaSuccess) rc = QST_ERR_CUDA;
                for (size_t j = 0; j < L.size() && !rc; ++j) batch_launch(b, *L[j], b->streams[j % ns]);
                for (int j = 0; j < used && !rc; ++j)
                    if (cudaEventRecord(b->join[j], b->streams[j]) != cudaSuccess ||
                        cudaStreamWaitEvent(cs, b->join[j], 0) != cudaSuccess)
                        rc = QST_ERR_CUDA;
            }
            if (!rc && cudaGetLastError() != cudaSuccess) rc = QST_ERR_CUDA;
        } else {
            for (int i = 0; i < b->count && !rc; ++i) {
                void *si = (void *)b->streams[i % ns];
                // qst_evaluate: with the instance plan's transform cache (two-round plans) the
                // adjoint applies only the inverse rounds
                rc = qst_evaluate(b->plans[i], psi[i], w[i], basis[i], row_ptr[i], outcome[i], count[i], shots[i],
                                  nullptr, c_obs[i], loss[i], grad_psi[i], grad_w[i], si);
            }
            for (int j = 0; j < ns && !rc; ++j)
                if (cudaEventRecord(b->join[j], b->streams[j]) != cudaSuccess ||
                    cudaStreamWaitEvent(cs, b->join[j], 0) != cudaSuccess)
                    rc = QST_ERR_CUDA;
        }
        const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
        if (rc || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rc ? rc : QST_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            b->exec = nullptr;
            return QST_ERR_CUDA;
        }
        b->key = key;
    }
    return cudaGraphLaunch(b->exec, st) == cudaSuccess ? QST_OK : QST_ERR_CUDA;
}

// Algorithm 1 on every instance of the batch: each instance's qst_iterate
// launch sequence (with its conditional trial nodes and device stopping
// rules) captured on its own forked stream into one CUDA graph, replayed on
// later calls with the same pointers, T, start and parameters.
extern "C" qst_status qst_batch_iterate(qst_batch b, int T, int t0, float *const *psi, float *const *w,
                                        const uint8_t *const *basis, const int64_t *const *row_ptr,
                                        const uint32_t *const *outcome, const uint32_t *const *count,
                                        const uint32_t *const *shots, const qst_iter_params *params,
                                        double *const *J_hist, int *const *accepted_hist, void *stream) {
    if (!b || T < 1 || t0 < 0 || !psi || !w || !basis || !row_ptr || !outcome || !count || !shots || !J_hist)
        return QST_ERR_INVALID_ARG;
    qst_iter_params ip;
    qst_iter_params_default(&ip);
    if (params) ip = *params;
    const qst_step_params &sp = ip.step;
    if (sp.n_eta < 1 || !(sp.eta0 > 0.0) || !(sp.eta_ratio > 0.0) || ip.T_alpha < 0 || ip.T_ref < 0 ||
        ip.delta_window < 0 || ip.delta_window >= kIterRing || !(ip.delta_tol >= 0.0) || ip.max_oracle_calls < 0 ||
        ip.spectral != 0)
        return QST_ERR_INVALID_ARG;
    std::vector<double> key = {(double)T, (double)(t0 == 0), sp.mu, sp.tau, sp.tau_acc, sp.eta0, sp.eta_ratio,
                               (double)sp.n_eta, (double)ip.T_alpha, (double)ip.T_ref, (double)ip.delta_window,
                               ip.delta_tol, (double)ip.max_oracle_calls};
    for (int t = 0; t < T; ++t) key.push_back((double)iter_slot(ip, (int64_t)t0 + t));
    for (int i = 0; i < b->count; ++i) {
        const qst_plan p = b->plans[i];
        if (!psi[i] || !w[i] || !basis[i] || !row_ptr[i] || !shots[i] || !J_hist[i]) return QST_ERR_INVALID_ARG;
        if (p->nnz > 0 && (!outcome[i] || !count[i])) return QST_ERR_INVALID_ARG;
        if (!aligned(psi[i], 16) || !aligned(w[i], 4) || !aligned(J_hist[i], 8) ||
            (accepted_hist && accepted_hist[i] && !aligned(accepted_hist[i], 4)))
            return QST_ERR_INVALID_ARG;
        if (p->wide || p->K > kProjMax) return QST_ERR_UNSUPPORTED;
        for (int t = 0; t < T; ++t)
            if (iter_slot(ip, (int64_t)t0 + t) == 2 && !p->refac_C) return QST_ERR_UNSUPPORTED;
        const void *ptrs[10] = {psi[i], w[i], basis[i], row_ptr[i], outcome[i], count[i], shots[i], J_hist[i],
                                accepted_hist ? accepted_hist[i] : nullptr, nullptr};
        for (const void *q : ptrs) key.push_back((double)(uintptr_t)q);
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->it_exec || key != b->it_key) {
        if (b->it_exec) {
            cudaGraphExecDestroy(b->it_exec);
            b->it_exec = nullptr;
        }
        for (auto p : b->plans)
            if (!p->it_body && cudaStreamCreateWithFlags(&p->it_body, cudaStreamNonBlocking) != cudaSuccess)
                return QST_ERR_CUDA;
        cudaStream_t cs = b->cap;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return QST_ERR_CUDA;
        }
        qst_status rc = QST_OK;
        const int ns = (int)b->streams.size();
        if (cudaEventRecord(b->start, cs) != cudaSuccess) rc = QST_ERR_CUDA;
        for (int j = 0; j < ns && !rc; ++j)
            if (cudaStreamWaitEvent(b->streams[j], b->start, 0) != cudaSuccess) rc = QST_ERR_CUDA;
        std::vector<bool> timing(b->count);
        std::vector<int64_t> before(b->count);
        for (int i = 0; i < b->count && !rc; ++i) {
            const qst_plan p = b->plans[i];
            timing[i] = p->timing;
            before[i] = p->total_launches;
            p->timing = false;  // no event records inside the graph
            rc = iterate_sequence(p, T, t0, psi[i], w[i], basis[i], row_ptr[i], outcome[i], count[i], shots[i], ip,
                                  J_hist[i], accepted_hist ? accepted_hist[i] : nullptr, b->streams[i % ns]);
            p->timing = timing[i];
            p->it_launches = p->total_launches - before[i];
            p->total_launches = before[i];
        }
        for (int j = 0; j < ns && !rc; ++j)
            if (cudaEventRecord(b->join[j], b->streams[j]) != cudaSuccess ||
                cudaStreamWaitEvent(cs, b->join[j], 0) != cudaSuccess)
                rc = QST_ERR_CUDA;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
        if (rc || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rc ? rc : QST_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&b->it_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            b->it_exec = nullptr;
            return QST_ERR_CUDA;
        }
        b->it_key = key;
    }
    if (cudaGraphLaunch(b->it_exec, st) != cudaSuccess) return QST_ERR_CUDA;
    for (auto p : b->plans) p->total_launches += p->it_launches;
    return QST_OK;
}
