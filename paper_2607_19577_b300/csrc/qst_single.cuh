// Single-setting chunk kernels for the wide path (n = 17..20; included inside
// qst.cu's anonymous namespace, after qst_fixed.cuh).
//
// Every wide-path unit (setting j of a group, high pattern f, atom k) carries
// one setting, so there is nothing to amortise over settings: the kernels
// below build the source chunk straight into registers (round-0 layout of the
// fixed rounds), run the three fixed rounds, and write z (adjoint) or gather
// w |.|^2 (forward) from registers.  Compared with k_forward_fx / k_adjoint_fx
// on single-setting bins they drop the tensor-memory staging of the source and
// the accumulator, the cp.async staging of the outcomes, the clearing of the c
// buffer and one block barrier; the shared memory (exchange buffer + one float
// buffer, 52 KB) admits four CTAs per SM.

constexpr int kFx1Smem = (8 + 4) * kFxBuf;  // exchange buffer (complex64) + float buffer
static_assert(4 * (kFx1Smem + 1024) <= 228 * 1024, "four CTAs per SM");

// The unit's setting: masks, 2^-m and its outcomes in chunk f (CSR range).
struct Fx1Unit {
    uint32_t xy, y;
    float cs;
    int64_t lo;
    int cnt;
};
__device__ __forceinline__ Fx1Unit fx1_unit(const Bin &b, uint32_t f, int nf, const int32_t *__restrict__ order,
                                            const SetPlan *__restrict__ plans, const int64_t *__restrict__ row_ptr,
                                            const int32_t *__restrict__ choff) {
    const int s = order[b.start];
    const SetPlan &P = plans[s];
    Fx1Unit u;
    u.xy = P.xy;
    u.y = P.y;
    u.cs = exp2f(-(float)P.m);
    const int32_t c0 = choff[(size_t)s * nf + f], c1 = choff[(size_t)s * nf + f + 1];
    u.lo = row_ptr[s] + c0;
    u.cnt = c1 - c0;
    return u;
}

// Forward unit = (single-setting bin, high pattern f, atom k).  CACHE (the
// evaluate path with the transform cache): the round-2 values also go to the
// exchange buffer and the gather stores them, unscaled, at the observed
// outcomes into the atom's slice of a.phi_obs.
template <bool CACHE>
__global__ void __launch_bounds__(kFxT, 4) k_forward_fx1(const FwdArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *work = reinterpret_cast<float2 *>(smem);
    float *pbuf = reinterpret_cast<float *>(smem + 8 * kFxBuf);
    const uint32_t tid = threadIdx.x;
    const int unit = blockIdx.x;
    const int k = unit % a.K;
    const int rest = unit / a.K;
    const uint32_t f = rest & ((1u << a.r) - 1u);
    const int bin = rest >> a.r;
    if (bin >= *a.n_bins || (a.skip && *a.skip)) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    constexpr uint32_t cmask = 4095u;
    float2 v[16];  // the source loads go out before the setting's metadata chain
    {
        const float2 *psik = a.psi + (size_t)bin * a.src_bin_stride + (size_t)k * D;
        build_source_regs<12, 4, 0, 8>(v, psik, f, b.xytop, b.ytop, tid);
        build_source_regs<12, 4, 8, 8>(v, psik, f, b.xytop, b.ytop, tid);
    }
    const Fx1Unit us = fx1_unit(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff);
    const uint32_t b0 = fx_pidx(fx_ubase<0>(tid)), b1 = fx_pidx(fx_ubase<1>(tid)), b2 = fx_pidx(fx_ubase<2>(tid));
#pragma unroll
    for (int R = 0; R < 3; ++R) {
        butterfly_fwd<4>(v, fx_bits(us.xy, R), fx_bits(us.y, R));
        if (R < 2) fx_exchange(v, work, R, R + 1, b0, b1, b2);
    }
    const float sc = a.w[k] * us.cs;
#pragma unroll
    for (int i = 0; i < 16; ++i) pbuf[b2 + fx_roff<2>(i)] = sc * (v[i].x * v[i].x + v[i].y * v[i].y);
    if (CACHE) {
        __syncwarp();  // the warp's round-2 reads of the exchange buffer are done (fx_exchange's last load)
        fx_store<2>(v, work, b2);
    }
    __syncthreads();
    float *pk = a.ppart + (size_t)k * a.nnz;
    for (int j = tid; j < us.cnt; j += kFxT) {
        const uint32_t u = a.outcome[us.lo + j] & cmask;
        pk[us.lo + j] = pbuf[fx_pidx(u)];
        if (CACHE) a.phi_obs[(size_t)k * a.nnz + us.lo + j] = work[fx_pidx(u)];
    }
    if (a.p_dense) {
        const int s = a.order[b.start];
        float *pd = a.p_dense + (size_t)s * D + ((size_t)f << 12);
        for (uint32_t u = tid; u <= cmask; u += kFxT) atomicAdd(pd + u, pbuf[fx_pidx(u)]);
    }
}

// Adjoint unit = (single-setting bin, high pattern f, atom k): zero the dense
// c buffer, scatter c 2^-m, forward rounds 0, 1, 2 (the first block barrier
// publishes the scatter), the c multiply, inverse rounds 2, 1, 0, and z from
// registers (round-0 layout).
__global__ void __launch_bounds__(kFxT, 4) k_adjoint_fx1(const AdjArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *work = reinterpret_cast<float2 *>(smem);
    float *cden = reinterpret_cast<float *>(smem + 8 * kFxBuf);
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
    float2 v[16];  // the source loads go out before the setting's metadata chain
    {
        const float2 *psik = a.psi + (size_t)bin * a.src_bin_stride + (size_t)k * D;
        build_source_regs<12, 4, 0, 8>(v, psik, f, b.xytop, b.ytop, tid);
        build_source_regs<12, 4, 8, 8>(v, psik, f, b.xytop, b.ytop, tid);
    }
    const Fx1Unit us = fx1_unit(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff);
    for (int u = tid; u < kFxBuf; u += kFxT) cden[u] = 0.f;
    __syncthreads();  // the buffer is zeroed before any entry is scattered
    for (int j = tid; j < us.cnt; j += kFxT)
        cden[fx_pidx(a.outcome[us.lo + j] & cmask)] = a.c_obs[us.lo + j] * us.cs;
    const uint32_t b0 = fx_pidx(fx_ubase<0>(tid)), b1 = fx_pidx(fx_ubase<1>(tid)), b2 = fx_pidx(fx_ubase<2>(tid));
#pragma unroll
    for (int R = 0; R < 3; ++R) {
        butterfly_fwd<4>(v, fx_bits(us.xy, R), fx_bits(us.y, R));
        if (R < 2) fx_exchange(v, work, R, R + 1, b0, b1, b2);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float cc = cden[b2 + fx_roff<2>(i)];
        v[i].x *= cc;
        v[i].y *= cc;
    }
#pragma unroll
    for (int R = 2; R >= 0; --R) {
        butterfly_inv<4>(v, fx_bits(us.xy, R), fx_bits(us.y, R));
        if (R > 0) fx_exchange(v, work, R, R - 1, b0, b1, b2);
    }
    float2 *zo = a.zbuf + ((size_t)bin * a.K + k) * D + ((size_t)f << 12);
#pragma unroll
    for (int i = 0; i < 16; ++i) zo[tid + (i << 8)] = v[i];
}

// Cached adjoint unit (the evaluate path with the transform cache): the
// forward stored the setting's chunk transform phi at its observed outcomes,
// so y = c 2^-m phi is scattered into the zeroed exchange buffer, loaded in
// round 2's layout, and only the inverse rounds 2, 1, 0 run; z from registers
// (round-0 layout) over the group's intermediate, as k_adjoint_fx1 writes it.
// No source is built and the group's high pass before the adjoint is skipped.
__global__ void __launch_bounds__(kFxT, 4) k_adjoint_fx1c(const AdjArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *work = reinterpret_cast<float2 *>(smem);
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
    const Fx1Unit us = fx1_unit(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff);
    for (int u = tid; u < kFxBuf; u += kFxT) work[u] = make_float2(0.f, 0.f);
    __syncthreads();  // zeroed before any entry is scattered
    const float2 *phk = a.phi_obs + (size_t)k * a.nnz;
    for (int j = tid; j < us.cnt; j += kFxT) {
        const float cy = a.c_obs[us.lo + j] * us.cs;
        const float2 ph = phk[us.lo + j];
        work[fx_pidx(a.outcome[us.lo + j] & cmask)] = make_float2(cy * ph.x, cy * ph.y);
    }
    __syncthreads();  // the scatter is visible
    const uint32_t b0 = fx_pidx(fx_ubase<0>(tid)), b1 = fx_pidx(fx_ubase<1>(tid)), b2 = fx_pidx(fx_ubase<2>(tid));
    float2 v[16];
    fx_load<2>(v, work, b2);
#pragma unroll
    for (int R = 2; R >= 0; --R) {
        butterfly_inv<4>(v, fx_bits(us.xy, R), fx_bits(us.y, R));
        if (R > 0) fx_exchange(v, work, R, R - 1, b0, b1, b2);
    }
    float2 *zo = a.zbuf + ((size_t)bin * a.K + k) * D + ((size_t)f << 12);
#pragma unroll
    for (int i = 0; i < 16; ++i) zo[tid + (i << 8)] = v[i];
}
