// Warp-per-unit chunk kernels for states of 5..9 qubits (included inside
// qst.cu's anonymous namespace, after qst_tworound.cuh).
//
// When the whole state is one chunk (r = 0) and small, a CTA per (bin, atom)
// leaves most of a warp idle (2^(n-4) threads at n <= 9).  Here a warp is the
// unit: lane l holds amplitudes u = 32 e + l, e < E = 2^(n-5), so the
// butterflies on outcome bits 5.. are in registers (the Hermitian chunk
// factors of the two-round kernels) and those on bits 0..4 pair lanes by
// shuffles.  A warp runs its bin's settings for one atom in order; four
// warps (four units) share a CTA only for scheduling, with no barrier
// between them.
//
// Lane-bit factor on bit j, own value v, partner's value o, s = +1 on the
// lane with bit j clear (it holds the first element a) and -1 on the other:
//   X: (a, b) -> (a + b, a - b)          new v = o + s v
//   Y: (a, b) -> (a - i b, i a - b)      new v = s (v + (Im o, -Re o))
// (both cases checked against the in-register butterflies: for s = -1 the Y
// row gives i a - b = -(b + (Im a, -Re a)) with a = o.)

constexpr int kWuT = 128;         // threads per CTA: four units
constexpr int kWuMaxQubits = 9;   // largest state run by warp units

// The chunk transform of one setting (it is its own inverse up to 2^m).
template <int NB>
__device__ __forceinline__ void wu_transform(float2 (&v)[1 << (NB - 5)], uint32_t xy, uint32_t y, uint32_t lane) {
    constexpr int E = 1 << (NB - 5);
    butterfly_herm<NB - 5>(v, xy >> 5, y >> 5);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        if (!((xy >> j) & 1u)) continue;  // warp-uniform
        const float s = ((lane >> j) & 1u) ? -1.f : 1.f;
        if ((y >> j) & 1u) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float ox = __shfl_xor_sync(0xffffffffu, v[e].x, 1 << j);
                const float oy = __shfl_xor_sync(0xffffffffu, v[e].y, 1 << j);
                v[e].x = s * __fadd_rn(v[e].x, oy);
                v[e].y = s * __fsub_rn(v[e].y, ox);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float ox = __shfl_xor_sync(0xffffffffu, v[e].x, 1 << j);
                const float oy = __shfl_xor_sync(0xffffffffu, v[e].y, 1 << j);
                v[e].x = __fmaf_rn(s, v[e].x, ox);
                v[e].y = __fmaf_rn(s, v[e].y, oy);
            }
        }
    }
}

// Forward unit = (bin, atom): per setting, w_k 2^-m |(V_s psi_k)_u|^2 into the
// warp's float buffer, then gathered at the setting's observed outcomes into
// the atom's slice of the partial buffer (and added into p_dense if given).
template <int NB>
__device__ __forceinline__ void forward_wu_body(const FwdArgs a, const int cta) {
    constexpr int E = 1 << (NB - 5), D = 1 << NB;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    float *pbuf = reinterpret_cast<float *>(smem) + warp * D;
    const int unit = cta * (kWuT / 32) + (int)warp;
    const int k = unit % a.K, bin = unit / a.K;
    if (bin >= *a.n_bins || (a.skip && *a.skip)) return;
    const Bin b = a.bins[bin];
    const float2 *psik = a.psi + (size_t)k * D;
    const float wk = a.w[k];
    float *pk = a.ppart + (size_t)k * a.nnz;
    for (int si = 0; si < b.count; ++si) {
        const int s = a.order[b.start + si];
        const SetPlan &P = a.plans[s];
        const uint32_t xy = P.xy, yy = P.y;
        const float sc = wk * exp2f(-(float)P.m);
        const int64_t lo = a.row_ptr[s] + a.choff[2 * s];
        const int cnt = a.choff[2 * s + 1] - a.choff[2 * s];
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = __ldg(psik + 32 * e + lane);
        wu_transform<NB>(v, xy, yy, lane);
#pragma unroll
        for (int e = 0; e < E; ++e) pbuf[32 * e + lane] = scaled_abs2(sc, v[e]);
        __syncwarp();
        for (int j = (int)lane; j < cnt; j += 32) pk[lo + j] = pbuf[a.outcome[lo + j] & (uint32_t)(D - 1)];
        if (a.p_dense) {
            float *pd = a.p_dense + (size_t)s * D;
#pragma unroll
            for (int e = 0; e < E; ++e) atomicAdd(pd + 32 * e + lane, pbuf[32 * e + lane]);
        }
        __syncwarp();  // the gather is done before the next setting overwrites the buffer
    }
}
template <int NB>
__global__ void __launch_bounds__(kWuT) k_forward_wu(const FwdArgs a) {
    forward_wu_body<NB>(a, blockIdx.x);
}
template <int NB>
__global__ void __launch_bounds__(kWuT) k_forward_wu_multi(const FwdArgs *__restrict__ args,
                                                          const int *__restrict__ start, int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const FwdArgs a = args[i];
    forward_wu_body<NB>(a, (int)blockIdx.x - start[i]);
}

// Adjoint unit = (bin, atom): per setting, the dense c 2^-m (zero where not
// observed) in the warp's float buffer, the transform of psi_k, the product,
// the inverse transform (the same factors), added into the register
// accumulator; z written once per unit.
template <int NB>
__device__ __forceinline__ void adjoint_wu_body(const AdjArgs a, const int cta) {
    if (a.skip && *a.skip) return;
    constexpr int E = 1 << (NB - 5), D = 1 << NB;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    float *cden = reinterpret_cast<float *>(smem) + warp * D;
    const int unit = cta * (kWuT / 32) + (int)warp;
    const int k = unit % a.K, bin = unit / a.K;
    if (bin >= *a.n_bins) return;
    const Bin b = a.bins[bin];
    const float2 *psik = a.psi + (size_t)k * D;
    float2 z[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        z[e] = make_float2(0.f, 0.f);
        cden[32 * e + lane] = 0.f;
    }
    for (int si = 0; si < b.count; ++si) {
        const int s = a.order[b.start + si];
        const SetPlan &P = a.plans[s];
        const uint32_t xy = P.xy, yy = P.y;
        const float cs = exp2f(-(float)P.m);
        const int64_t lo = a.row_ptr[s] + a.choff[2 * s];
        const int cnt = a.choff[2 * s + 1] - a.choff[2 * s];
        __syncwarp();  // the previous setting's clears are done
        for (int j = (int)lane; j < cnt; j += 32) cden[a.outcome[lo + j] & (uint32_t)(D - 1)] = a.c_obs[lo + j] * cs;
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = __ldg(psik + 32 * e + lane);
        wu_transform<NB>(v, xy, yy, lane);
        __syncwarp();  // the scatter is visible
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float c = cden[32 * e + lane];
            v[e].x = __fmul_rn(v[e].x, c);
            v[e].y = __fmul_rn(v[e].y, c);
        }
        wu_transform<NB>(v, xy, yy, lane);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            z[e].x = __fadd_rn(z[e].x, v[e].x);
            z[e].y = __fadd_rn(z[e].y, v[e].y);
        }
        __syncwarp();  // every lane has read its c values
        for (int j = (int)lane; j < cnt; j += 32) cden[a.outcome[lo + j] & (uint32_t)(D - 1)] = 0.f;
    }
    float2 *zo = a.zbuf + ((size_t)bin * a.K + k) * D;
#pragma unroll
    for (int e = 0; e < E; ++e) zo[32 * e + lane] = z[e];
}
template <int NB>
__global__ void __launch_bounds__(kWuT) k_adjoint_wu(const AdjArgs a) {
    adjoint_wu_body<NB>(a, blockIdx.x);
}
template <int NB>
__global__ void __launch_bounds__(kWuT) k_adjoint_wu_multi(const AdjArgs *__restrict__ args,
                                                          const int *__restrict__ start, int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const AdjArgs a = args[i];
    adjoint_wu_body<NB>(a, (int)blockIdx.x - start[i]);
}

// Shared memory of a warp-unit CTA: one float buffer of 2^n per warp.
constexpr int wu_smem(int nb) { return (kWuT / 32) * (1 << nb) * 4; }

// Calls fn(integral_constant<NB>) for a plan's state size (5..9 qubits).
template <typename Fn>
void with_wu(int nb, Fn &&fn) {
    switch (nb) {
        case 5: fn(std::integral_constant<int, 5>()); break;
        case 6: fn(std::integral_constant<int, 6>()); break;
        case 7: fn(std::integral_constant<int, 7>()); break;
        case 8: fn(std::integral_constant<int, 8>()); break;
        default: fn(std::integral_constant<int, 9>()); break;
    }
}
