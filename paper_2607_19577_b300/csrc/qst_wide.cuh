// qst_wide.cuh — the wide path (n = 17..20): the chunk is the low c = n - 8
// outcome bits, the high part always kWideR = 8 bits.  Binning by the high
// pattern would leave about one setting per bin at these sizes, so the high
// factor is applied with butterflies instead (over tiles of 256 rows x 32
// columns, each tile of psi read once per group), per group of settings and
// all atoms at once, so that each launch is large:
//   T[j][k] = (U_H(s_j) (x) I) psi_k                 k_high_fwd
//   chunk kernels on T (single-setting bins)         k_forward / k_adjoint
//   acc_k += sum_j (U_H(s_j)^* (x) I) Z[j][k]        k_high_inv_acc (FP64)
// Included by qst.cu inside its anonymous namespace.
#pragma once

constexpr int kWideR = 8;            // high bits of the wide path
constexpr int kWideCols = 32;        // columns per high-pass tile (256-byte rows)
constexpr int kWideT = 16 * kWideCols;  // threads per high-pass CTA: 16 row groups x the columns
constexpr int kWideSmem = 256 * kWideCols * (int)sizeof(float2);  // one 256-row tile (64 KB)
constexpr int kWideInvSmem = 2 * kWideSmem;                        // two tiles (the inverse pass)
constexpr int64_t kWideGroupBytes = 2048ll << 20;  // intermediate per group (all atoms of G settings)

// Forward high pass: T[j][k] = (U_H(s_j) (x) I) psi_k for every setting
// s_j = g0 + j of the group (grid: x = column tiles, y = atom k).  The CTA
// reads its 256-row tile of psi_k once and keeps it in registers while it
// loops over the settings.  Thread t: column t % 32; round 1 holds the rows
// (t / 32) * 16 + i (row bits 0..3 in registers), round 2 the rows
// i * 16 + t / 32 (row bits 4..7); a shared-memory transpose between them.
__global__ void __launch_bounds__(kWideT) k_high_fwd(const float2 *__restrict__ psi, const SetPlan *__restrict__ plans,
                                                     int g0, int G, int K, int c, float2 *__restrict__ T) {
    extern __shared__ __align__(16) unsigned char wide_smem[];
    float2 *tile = reinterpret_cast<float2 *>(wide_smem);
    const int k = blockIdx.y;
    const int col0 = blockIdx.x * kWideCols;
    const int t = threadIdx.x, l = t % kWideCols, q = t / kWideCols;
    const float2 *pk = psi + ((size_t)k << (c + kWideR));
    float2 src[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) src[i] = pk[((size_t)((q << 4) | i) << c) + col0 + l];
    for (int j = 0; j < G; ++j) {
        const int s = g0 + j;
        const uint32_t xyH = plans[s].xy >> c, yH = plans[s].y >> c;
        float2 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = src[i];
        butterfly_fwd<4>(v, xyH & 15u, yH & 15u);
        if (j > 0) __syncthreads();  // the previous setting's reads of the tile are done
#pragma unroll
        for (int i = 0; i < 16; ++i) tile[(((q << 4) | i) * kWideCols) + l] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = tile[(((i << 4) | q) * kWideCols) + l];
        butterfly_fwd<4>(v, (xyH >> 4) & 15u, (yH >> 4) & 15u);
        float2 *Tj = T + (((size_t)j * K + k) << (c + kWideR));
#pragma unroll
        for (int i = 0; i < 16; ++i) Tj[((size_t)((i << 4) | q) << c) + col0 + l] = v[i];
    }
}

// Inverse high pass with accumulation: acc_k += sum_{j < G} (U_H(s_j)^* (x) I) Z[j][k]
// for the settings s_j = g0 + j (grid: x = column tiles, y = atom k).  The
// group's sum is compensated (Kahan) FP32 in registers -- B300's FP64 rate is
// a few operations per SM cycle, too slow for a per-setting FP64 add -- and
// is folded into the FP64 accumulator once per group.  The Z tiles stream through two shared-memory buffers with
// cp.async (tile j + 2 loads while tile j is transformed); each landed buffer
// also serves as the transpose between the two rounds.
__global__ void __launch_bounds__(kWideT) k_high_inv_acc(const float2 *__restrict__ Z, const SetPlan *__restrict__ plans,
                                                         int g0, int G, int K, int c, double2 *__restrict__ acc) {
    extern __shared__ __align__(16) unsigned char wide_smem[];
    float2 *buf = reinterpret_cast<float2 *>(wide_smem);  // [2][256 rows][kWideCols]
    const int col0 = blockIdx.x * kWideCols;
    const int k = blockIdx.y;
    const int t = threadIdx.x, l = t % kWideCols, q = t / kWideCols;
    constexpr int kPieces = 256 * kWideCols / 2;  // 16-byte pieces of a tile
    // stage tile j into buffer j % 2 (or commit an empty group past the end)
    auto stage = [&](int j) {
        if (j < G) {
            const float2 *Zj = Z + (((size_t)j * K + k) << (c + kWideR)) + col0;
            float2 *dst = buf + (size_t)(j & 1) * 256 * kWideCols;
            for (int e = t; e < kPieces; e += kWideT) {
                const int row = e / (kWideCols / 2), piece = e % (kWideCols / 2);
                const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + row * kWideCols + 2 * piece);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa),
                             "l"(Zj + ((size_t)row << c) + 2 * piece)
                             : "memory");
            }
        }
        cp_async_commit();
    };
    float2 a[16], e[16];  // running sum and its Kahan compensation (true sum = a - e)
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = e[i] = make_float2(0.f, 0.f);
    stage(0);
    stage(1);
    for (int j = 0; j < G; ++j) {
        const int s = g0 + j;
        const uint32_t xyH = plans[s].xy >> c, yH = plans[s].y >> c;
        float2 *tile = buf + (size_t)(j & 1) * 256 * kWideCols;
        cp_async_wait1();  // this thread's pieces of tile j have landed
        __syncthreads();   // and everyone's
        float2 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = tile[(((i << 4) | q) * kWideCols) + l];
        butterfly_inv<4>(v, (xyH >> 4) & 15u, (yH >> 4) & 15u);
#pragma unroll
        for (int i = 0; i < 16; ++i) tile[(((i << 4) | q) * kWideCols) + l] = v[i];  // the addresses just read
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = tile[(((q << 4) | i) * kWideCols) + l];
        butterfly_inv<4>(v, xyH & 15u, yH & 15u);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float yx = v[i].x - e[i].x, yy = v[i].y - e[i].y;
            const float tx = a[i].x + yx, ty = a[i].y + yy;
            e[i].x = (tx - a[i].x) - yx;
            e[i].y = (ty - a[i].y) - yy;
            a[i] = make_float2(tx, ty);
        }
        __syncthreads();  // every read of this buffer is done before it is refilled
        stage(j + 2);
    }
    cp_async_wait0();
    double2 *ak = acc + ((size_t)k << (c + kWideR));
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        double2 *p = ak + ((size_t)((q << 4) | i) << c) + col0 + l;
        const double2 o = *p;
        *p = make_double2(o.x + ((double)a[i].x - (double)e[i].x), o.y + ((double)a[i].y - (double)e[i].y));
    }
}

// Single-setting bins g0 .. g0 + G - 1 for the chunk kernels of one group.
__global__ void k_wide_bins(int g0, int G, Bin *__restrict__ bins, int *__restrict__ n_bins) {
    for (int j = threadIdx.x; j < G; j += blockDim.x) {
        Bin b;
        b.start = g0 + j;
        b.count = 1;
        b.xytop = 0;
        b.ytop = 0;
        bins[j] = b;
    }
    if (threadIdx.x == 0) *n_bins = G;
}

// grad_k = -(w_k / B) acc_k (FP32 out), and per-thread FP64 partials of
// Re <psi_k, acc_k> for h_k (summed by k_hsum).  Thread per (k, low index l),
// looping over the 2^8 high rows.
__global__ void __launch_bounds__(256) k_wide_final(const double2 *__restrict__ acc, const float *__restrict__ w,
                                                    const float2 *__restrict__ psi, float2 *__restrict__ grad,
                                                    double *__restrict__ hdot, int n, int c, int K, float invB) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ((int64_t)K << c)) return;
    const int k = (int)(idx >> c);
    const uint32_t l = (uint32_t)(idx & ((1 << c) - 1));
    const size_t base = ((size_t)k << n) + l;
    const double sc = -(double)w[k] * (double)invB;
    double hd = 0.0;
    for (int f = 0; f < (1 << kWideR); ++f) {
        const size_t e = base + ((size_t)f << c);
        const double2 g = acc[e];
        const float2 q = psi[e];
        grad[e] = make_float2((float)(sc * g.x), (float)(sc * g.y));
        hd += (double)q.x * g.x + (double)q.y * g.y;
    }
    hdot[idx] = hd;
}
