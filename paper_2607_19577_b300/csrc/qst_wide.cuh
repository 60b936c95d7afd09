// qst_wide.cuh — the wide path (n = 17..20): the chunk is the low c = n - 8
// outcome bits, the high part always kWideR = 8 bits.  Binning by the high
// pattern would leave about one setting per bin at these sizes, so the high
// factor is applied with butterflies instead (one pass per setting and atom,
// over tiles of 256 rows x 16 columns), per group of settings
// and all atoms at once, so that each launch is large:
//   T[j][k] = (U_H(s_j) (x) I) psi_k                 k_high_fwd
//   chunk kernels on T (single-setting bins)         k_forward / k_adjoint
//   acc_k += sum_j (U_H(s_j)^* (x) I) Z[j][k]        k_high_inv_acc (FP64)
// Included by qst.cu inside its anonymous namespace.
#pragma once

constexpr int kWideR = 8;            // high bits of the wide path
constexpr int kWideCols = 16;        // columns per high-pass tile (128-byte rows)
constexpr int64_t kWideGroupBytes = 512ll << 20;  // intermediate per group (all atoms of G settings)

// Forward high pass: T[j][k] = (U_H(s_j) (x) I) psi_k for the group's settings
// s_j = g0 + j (grid: x = column tiles, y = j, z = atom k).  Thread t:
// column t & 15; round 1 holds the rows (t >> 4) << 4 | i (row bits 0..3 in
// registers), round 2 the rows i << 4 | (t >> 4) (row bits 4..7); a
// shared-memory transpose between them.
__global__ void __launch_bounds__(256) k_high_fwd(const float2 *__restrict__ psi, const SetPlan *__restrict__ plans,
                                                  int g0, int K, int c, float2 *__restrict__ T) {
    __shared__ float2 tile[256 * kWideCols];
    const int j = blockIdx.y, k = blockIdx.z;
    const int s = g0 + j;
    const int col0 = blockIdx.x * kWideCols;
    const uint32_t xyH = plans[s].xy >> c, yH = plans[s].y >> c;
    const int t = threadIdx.x, l = t & 15, q = t >> 4;
    const float2 *pk = psi + ((size_t)k << (c + kWideR));
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = pk[((size_t)((q << 4) | i) << c) + col0 + l];
    butterfly_fwd<4>(v, xyH & 15u, yH & 15u);
#pragma unroll
    for (int i = 0; i < 16; ++i) tile[(((q << 4) | i) << 4) + l] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = tile[(((i << 4) | q) << 4) + l];
    butterfly_fwd<4>(v, (xyH >> 4) & 15u, (yH >> 4) & 15u);
    float2 *Tj = T + (((size_t)j * K + k) << (c + kWideR));
#pragma unroll
    for (int i = 0; i < 16; ++i) Tj[((size_t)((i << 4) | q) << c) + col0 + l] = v[i];
}

// Inverse high pass with accumulation: acc_k += sum_{j < G} (U_H(s_j)^* (x) I) Z[j][k]
// for the settings s_j = g0 + j; FP64 accumulation in registers over the
// group, one read-modify-write of acc per group (grid: x = column tiles,
// y = atom k).
__global__ void __launch_bounds__(256) k_high_inv_acc(const float2 *__restrict__ Z, const SetPlan *__restrict__ plans,
                                                      int g0, int G, int K, int c, double2 *__restrict__ acc) {
    __shared__ float2 tile[256 * kWideCols];
    const int col0 = blockIdx.x * kWideCols;
    const int k = blockIdx.y;
    const int t = threadIdx.x, l = t & 15, q = t >> 4;
    double2 a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = make_double2(0.0, 0.0);
    for (int j = 0; j < G; ++j) {
        const int s = g0 + j;
        const uint32_t xyH = plans[s].xy >> c, yH = plans[s].y >> c;
        const float2 *Zj = Z + (((size_t)j * K + k) << (c + kWideR));
        float2 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = Zj[((size_t)((i << 4) | q) << c) + col0 + l];
        butterfly_inv<4>(v, (xyH >> 4) & 15u, (yH >> 4) & 15u);
        __syncthreads();  // the previous setting's reads of the tile are done
#pragma unroll
        for (int i = 0; i < 16; ++i) tile[(((i << 4) | q) << 4) + l] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = tile[(((q << 4) | i) << 4) + l];
        butterfly_inv<4>(v, xyH & 15u, yH & 15u);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            a[i].x += (double)v[i].x;
            a[i].y += (double)v[i].y;
        }
    }
    double2 *ak = acc + ((size_t)k << (c + kWideR));
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        double2 *p = ak + ((size_t)((q << 4) | i) << c) + col0 + l;
        const double2 o = *p;
        *p = make_double2(o.x + a[i].x, o.y + a[i].y);
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
