// Packed-FP32 adjoint for 12-qubit chunks in two 6-qubit rounds (included
// inside qst.cu's anonymous namespace, after qst_tworound.cuh, whose round
// layout, CTA shape and setting staging it shares).
//
// The adjoint is bound by instruction issue, not by the FP32 pipe, and
// sm_103a executes a pair of FP32 operations held in one 64-bit register
// (add/sub/mul/fma .f32x2) as one instruction at the full lane rate.  A
// thread's 64 amplitudes are therefore held as 32 + 32 packed registers:
//   X[p] = (Re v[p], Re v[p + 32]),  Y[p] = (Im v[p], Im v[p + 32]),  p < 32,
// so a butterfly on element bit j < 5 pairs X[p] with X[p | 2^j] (and the Y
// registers alike) and needs 4 packed instructions for two complex pairs
// instead of 8 scalar ones; element bit 5 pairs the two halves of each
// register and runs on scalar halves.  (The forward kernel stays on scalar
// registers: with packed registers it needs about 190 registers, which costs
// it a third of its warps per SM, and measured slower.)
//
// Exchange buffers (one per atom): two float planes (real, imaginary), 64
// rows (hi) of 68 floats; lo sits at column col(lo) = 2 (lo mod 32) + lo / 32,
// so lo and lo + 32 are adjacent and a round-B thread reads and writes its row
// as 16-byte vectors (two packed registers per plane).  A round-A thread owns
// one column: thread t holds lo(t) = (t mod 32) / 2 + 16 (t / 32) + 32 (t mod
// 2), so the 32 lanes of a warp write 32 consecutive words of a row (one
// scalar access per half register, conflict-free); the 68-float rows put the
// 8 lanes of a quarter-warp's 16-byte accesses on distinct bank groups.  The
// dense c buffers use the same positions.

typedef unsigned long long f2p;  // two FP32 values in one 64-bit register (low word = first)
__device__ __forceinline__ f2p p_add(f2p a, f2p b) {
    f2p d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p p_sub(f2p a, f2p b) {
    f2p d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p p_mul(f2p a, f2p b) {
    f2p d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// a * b + c, one rounding per element
__device__ __forceinline__ f2p p_fma(f2p a, f2p b, f2p c) {
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ void p_unpack(f2p a, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}
constexpr f2p kM2 = 0xC0000000C0000000ull;   // (-2, -2)

constexpr int k2pPR = 68;                 // floats per row of a plane
constexpr int k2pPlane = 64 * k2pPR;      // floats of one plane (also one dense c buffer)
constexpr int k2pBuf = 2 * k2pPlane;      // floats of one atom's exchange buffer (real + imaginary plane)
constexpr uint32_t k2ColsAdj = 256;          // TMEM columns of an adjoint CTA: source + accumulator

// column of lo in a plane row; plane position of chunk index u
__host__ __device__ constexpr uint32_t k2p_col(uint32_t lo) { return 2u * (lo & 31u) + (lo >> 5); }
__host__ __device__ constexpr uint32_t k2p_pos(uint32_t u) { return (u >> 6) * (uint32_t)k2pPR + k2p_col(u & 63u); }
// lo owned by thread t (0..63 within its atom) in round A
__device__ __forceinline__ uint32_t k2p_lo(uint32_t t) { return ((t & 31u) >> 1) + 16u * (t >> 5) + 32u * (t & 1u); }

// Adjoint CTA: the two atoms' exchange buffers, two dense c buffers (settings
// alternate, shared by both atoms), the staged (outcome, c) pairs of two
// settings, the bin's masks and metadata, the TMEM address.
__host__ __device__ constexpr K2Smem k2p_smem() {
    K2Smem sp{};
    sp.work = 0;
    sp.fbuf = sp.work + 2 * k2pBuf * 4;
    sp.stage = sp.fbuf + 2 * k2pPlane * 4;
    sp.masks = sp.stage + 2 * k2Stage * 8;
    sp.meta = sp.masks + kMaxBin * (int)sizeof(uint2);
    sp.tmem = sp.meta + kMaxBin * (int)sizeof(SetMeta);
    sp.total = sp.tmem + 16;
    return sp;
}
static_assert(k2p_smem().fbuf % 16 == 0 && k2p_smem().stage % 16 == 0 && k2p_smem().masks % 16 == 0 &&
                  k2p_smem().meta % 16 == 0,
              "aligned shared arrays");
static_assert((k2pPR * 4) % 16 == 0, "plane rows are 16-byte aligned");
constexpr int k2CtaAdj = k2p_smem().total + 1024;
static_assert(2 * k2CtaAdj <= k2SmemSM, "two adjoint CTAs per SM");
// Shared memory admits at most two adjoint CTAs, three forward CTAs, or one
// of each, on an SM; their TMEM columns then fit in the SM's 512, so an
// allocation never waits (forward and adjoint CTAs of different instances
// can share an SM when the batched graph runs them concurrently).
static_assert(3 * k2CtaAdj > k2SmemSM && k2CtaAdj + 2 * k2CtaFwd > k2SmemSM && 2 * k2ColsAdj <= 512 &&
                  3 * k2ColsFwd <= 512 && k2ColsAdj + k2ColsFwd <= 512,
              "TMEM never oversubscribed");

// Tensor-memory image of a thread's 64 amplitudes: columns 0..63 hold the X
// registers (X[p] in columns 2p, 2p + 1), columns 64..127 the Y registers, so
// each 32-column load fills 16 packed registers in register order.  The
// 32-bit halves stay inside the asm blocks, so the packed registers are
// loaded and stored in place.
__device__ __forceinline__ void k2p_tm_ld(uint32_t taddr, f2p (&X)[32], f2p (&Y)[32]) {
    asm volatile(
        "{\n\t.reg .b32 r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15,r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31,r32,r33,r34,r35,r36,r37,r38,r39,r40,r41,r42,r43,r44,r45,r46,r47,r48,r49,r50,r51,r52,r53,r54,r55,r56,r57,r58,r59,r60,r61,r62,r63,r64,r65,r66,r67,r68,r69,r70,r71,r72,r73,r74,r75,r76,r77,r78,r79,r80,r81,r82,r83,r84,r85,r86,r87,r88,r89,r90,r91,r92,r93,r94,r95,r96,r97,r98,r99,r100,r101,r102,r103,r104,r105,r106,r107,r108,r109,r110,r111,r112,r113,r114,r115,r116,r117,r118,r119,r120,r121,r122,r123,r124,r125,r126,r127;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15,r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31}, [%64];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {r32,r33,r34,r35,r36,r37,r38,r39,r40,r41,r42,r43,r44,r45,r46,r47,r48,r49,r50,r51,r52,r53,r54,r55,r56,r57,r58,r59,r60,r61,r62,r63}, [%65];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {r64,r65,r66,r67,r68,r69,r70,r71,r72,r73,r74,r75,r76,r77,r78,r79,r80,r81,r82,r83,r84,r85,r86,r87,r88,r89,r90,r91,r92,r93,r94,r95}, [%66];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {r96,r97,r98,r99,r100,r101,r102,r103,r104,r105,r106,r107,r108,r109,r110,r111,r112,r113,r114,r115,r116,r117,r118,r119,r120,r121,r122,r123,r124,r125,r126,r127}, [%67];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "mov.b64 %1, {r2, r3};\n\t"
        "mov.b64 %2, {r4, r5};\n\t"
        "mov.b64 %3, {r6, r7};\n\t"
        "mov.b64 %4, {r8, r9};\n\t"
        "mov.b64 %5, {r10, r11};\n\t"
        "mov.b64 %6, {r12, r13};\n\t"
        "mov.b64 %7, {r14, r15};\n\t"
        "mov.b64 %8, {r16, r17};\n\t"
        "mov.b64 %9, {r18, r19};\n\t"
        "mov.b64 %10, {r20, r21};\n\t"
        "mov.b64 %11, {r22, r23};\n\t"
        "mov.b64 %12, {r24, r25};\n\t"
        "mov.b64 %13, {r26, r27};\n\t"
        "mov.b64 %14, {r28, r29};\n\t"
        "mov.b64 %15, {r30, r31};\n\t"
        "mov.b64 %16, {r32, r33};\n\t"
        "mov.b64 %17, {r34, r35};\n\t"
        "mov.b64 %18, {r36, r37};\n\t"
        "mov.b64 %19, {r38, r39};\n\t"
        "mov.b64 %20, {r40, r41};\n\t"
        "mov.b64 %21, {r42, r43};\n\t"
        "mov.b64 %22, {r44, r45};\n\t"
        "mov.b64 %23, {r46, r47};\n\t"
        "mov.b64 %24, {r48, r49};\n\t"
        "mov.b64 %25, {r50, r51};\n\t"
        "mov.b64 %26, {r52, r53};\n\t"
        "mov.b64 %27, {r54, r55};\n\t"
        "mov.b64 %28, {r56, r57};\n\t"
        "mov.b64 %29, {r58, r59};\n\t"
        "mov.b64 %30, {r60, r61};\n\t"
        "mov.b64 %31, {r62, r63};\n\t"
        "mov.b64 %32, {r64, r65};\n\t"
        "mov.b64 %33, {r66, r67};\n\t"
        "mov.b64 %34, {r68, r69};\n\t"
        "mov.b64 %35, {r70, r71};\n\t"
        "mov.b64 %36, {r72, r73};\n\t"
        "mov.b64 %37, {r74, r75};\n\t"
        "mov.b64 %38, {r76, r77};\n\t"
        "mov.b64 %39, {r78, r79};\n\t"
        "mov.b64 %40, {r80, r81};\n\t"
        "mov.b64 %41, {r82, r83};\n\t"
        "mov.b64 %42, {r84, r85};\n\t"
        "mov.b64 %43, {r86, r87};\n\t"
        "mov.b64 %44, {r88, r89};\n\t"
        "mov.b64 %45, {r90, r91};\n\t"
        "mov.b64 %46, {r92, r93};\n\t"
        "mov.b64 %47, {r94, r95};\n\t"
        "mov.b64 %48, {r96, r97};\n\t"
        "mov.b64 %49, {r98, r99};\n\t"
        "mov.b64 %50, {r100, r101};\n\t"
        "mov.b64 %51, {r102, r103};\n\t"
        "mov.b64 %52, {r104, r105};\n\t"
        "mov.b64 %53, {r106, r107};\n\t"
        "mov.b64 %54, {r108, r109};\n\t"
        "mov.b64 %55, {r110, r111};\n\t"
        "mov.b64 %56, {r112, r113};\n\t"
        "mov.b64 %57, {r114, r115};\n\t"
        "mov.b64 %58, {r116, r117};\n\t"
        "mov.b64 %59, {r118, r119};\n\t"
        "mov.b64 %60, {r120, r121};\n\t"
        "mov.b64 %61, {r122, r123};\n\t"
        "mov.b64 %62, {r124, r125};\n\t"
        "mov.b64 %63, {r126, r127};\n\t"
        "}"
        : "=l"(X[0]), "=l"(X[1]), "=l"(X[2]), "=l"(X[3]), "=l"(X[4]), "=l"(X[5]), "=l"(X[6]), "=l"(X[7]), "=l"(X[8]), "=l"(X[9]), "=l"(X[10]), "=l"(X[11]), "=l"(X[12]), "=l"(X[13]), "=l"(X[14]), "=l"(X[15]), "=l"(X[16]), "=l"(X[17]), "=l"(X[18]), "=l"(X[19]), "=l"(X[20]), "=l"(X[21]), "=l"(X[22]), "=l"(X[23]), "=l"(X[24]), "=l"(X[25]), "=l"(X[26]), "=l"(X[27]), "=l"(X[28]), "=l"(X[29]), "=l"(X[30]), "=l"(X[31]), "=l"(Y[0]), "=l"(Y[1]), "=l"(Y[2]), "=l"(Y[3]), "=l"(Y[4]), "=l"(Y[5]), "=l"(Y[6]), "=l"(Y[7]), "=l"(Y[8]), "=l"(Y[9]), "=l"(Y[10]), "=l"(Y[11]), "=l"(Y[12]), "=l"(Y[13]), "=l"(Y[14]), "=l"(Y[15]), "=l"(Y[16]), "=l"(Y[17]), "=l"(Y[18]), "=l"(Y[19]), "=l"(Y[20]), "=l"(Y[21]), "=l"(Y[22]), "=l"(Y[23]), "=l"(Y[24]), "=l"(Y[25]), "=l"(Y[26]), "=l"(Y[27]), "=l"(Y[28]), "=l"(Y[29]), "=l"(Y[30]), "=l"(Y[31])
        : "r"(taddr), "r"(taddr + 32u), "r"(taddr + 64u), "r"(taddr + 96u)
        : "memory");
}
// 16 packed registers -> 32 consecutive columns
__device__ __forceinline__ void k2p_tm_st16(uint32_t taddr, const f2p *R) {
    asm volatile(
        "{\n\t.reg .b32 r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15,r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31;\n\t"
        "mov.b64 {r0, r1}, %1;\n\t"
        "mov.b64 {r2, r3}, %2;\n\t"
        "mov.b64 {r4, r5}, %3;\n\t"
        "mov.b64 {r6, r7}, %4;\n\t"
        "mov.b64 {r8, r9}, %5;\n\t"
        "mov.b64 {r10, r11}, %6;\n\t"
        "mov.b64 {r12, r13}, %7;\n\t"
        "mov.b64 {r14, r15}, %8;\n\t"
        "mov.b64 {r16, r17}, %9;\n\t"
        "mov.b64 {r18, r19}, %10;\n\t"
        "mov.b64 {r20, r21}, %11;\n\t"
        "mov.b64 {r22, r23}, %12;\n\t"
        "mov.b64 {r24, r25}, %13;\n\t"
        "mov.b64 {r26, r27}, %14;\n\t"
        "mov.b64 {r28, r29}, %15;\n\t"
        "mov.b64 {r30, r31}, %16;\n\t"
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15,r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31};\n\t"
        "}"
        ::"r"(taddr), "l"(R[0]), "l"(R[1]), "l"(R[2]), "l"(R[3]), "l"(R[4]), "l"(R[5]), "l"(R[6]), "l"(R[7]), "l"(R[8]), "l"(R[9]), "l"(R[10]), "l"(R[11]), "l"(R[12]), "l"(R[13]), "l"(R[14]), "l"(R[15])
        : "memory");
}
// 32 consecutive columns -> 16 packed registers (waits for the load)
__device__ __forceinline__ void k2p_tm_ld16(uint32_t taddr, f2p *R) {
    asm volatile(
        "{\n\t.reg .b32 r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15,r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {r0,r1,r2,r3,r4,r5,r6,r7,r8,r9,r10,r11,r12,r13,r14,r15,r16,r17,r18,r19,r20,r21,r22,r23,r24,r25,r26,r27,r28,r29,r30,r31}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "mov.b64 %1, {r2, r3};\n\t"
        "mov.b64 %2, {r4, r5};\n\t"
        "mov.b64 %3, {r6, r7};\n\t"
        "mov.b64 %4, {r8, r9};\n\t"
        "mov.b64 %5, {r10, r11};\n\t"
        "mov.b64 %6, {r12, r13};\n\t"
        "mov.b64 %7, {r14, r15};\n\t"
        "mov.b64 %8, {r16, r17};\n\t"
        "mov.b64 %9, {r18, r19};\n\t"
        "mov.b64 %10, {r20, r21};\n\t"
        "mov.b64 %11, {r22, r23};\n\t"
        "mov.b64 %12, {r24, r25};\n\t"
        "mov.b64 %13, {r26, r27};\n\t"
        "mov.b64 %14, {r28, r29};\n\t"
        "mov.b64 %15, {r30, r31};\n\t"
        "}"
        : "=l"(R[0]), "=l"(R[1]), "=l"(R[2]), "=l"(R[3]), "=l"(R[4]), "=l"(R[5]), "=l"(R[6]), "=l"(R[7]), "=l"(R[8]), "=l"(R[9]), "=l"(R[10]), "=l"(R[11]), "=l"(R[12]), "=l"(R[13]), "=l"(R[14]), "=l"(R[15])
        : "r"(taddr)
        : "memory");
}
// z += v for the 128 accumulator columns (packed adds), 32 columns at a time.
// The previous setting's stores to z complete first (their wait sits here, so
// they drain during that setting's rounds).
__device__ __forceinline__ void k2p_tm_acc(uint32_t taddr, const f2p (&X)[32], const f2p (&Y)[32]) {
    tm_wait_st();
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const f2p *A = (h < 2 ? X : Y) + 16 * (h & 1);
        f2p z[16];
        k2p_tm_ld16(taddr + 32u * h, z);
#pragma unroll
        for (int i = 0; i < 16; ++i) z[i] = p_add(z[i], A[i]);
        k2p_tm_st16(taddr + 32u * h, z);
    }
}

// Chunk f of (U_h (x) I) psi_k in round A's layout (element i of thread t =
// amplitude lo(t) + 64 i) -> TMEM columns 0..127 in the packed order, built
// for elements 8Q..8Q+7 and 32+8Q..32+8Q+7 (16 X and 16 Y columns) at a time.
// An inactive atom (k >= K) gets zeros.  C < 12: element i of thread lo is
// amplitude lo + 2^(C-6) i.
template <int C = 12>
__device__ __forceinline__ void k2p_build_source(uint32_t t_src, const float2 *psik, bool active, uint32_t f,
                                                uint32_t xytop, uint32_t ytop, uint32_t lo) {
    float2 acc[64];
#define QST_K2_PART(Q)                                                                                   \
    {                                                                                                    \
        if (active) {                                                                                    \
            build_source_regs<C, 6, 8 * (Q), 8>(acc, psik, f, xytop, ytop, lo);                          \
            build_source_regs<C, 6, 32 + 8 * (Q), 8>(acc, psik, f, xytop, ytop, lo);                     \
        } else {                                                                                         \
            _Pragma("unroll") for (int i = 0; i < 8; ++i) {                                              \
                acc[8 * (Q) + i] = make_float2(0.f, 0.f);                                                \
                acc[32 + 8 * (Q) + i] = make_float2(0.f, 0.f);                                           \
            }                                                                                            \
        }                                                                                                \
        uint32_t rx[16], ry[16];                                                                         \
        _Pragma("unroll") for (int i = 0; i < 8; ++i) {                                                  \
            rx[2 * i] = __float_as_uint(acc[8 * (Q) + i].x);                                             \
            rx[2 * i + 1] = __float_as_uint(acc[32 + 8 * (Q) + i].x);                                    \
            ry[2 * i] = __float_as_uint(acc[8 * (Q) + i].y);                                             \
            ry[2 * i + 1] = __float_as_uint(acc[32 + 8 * (Q) + i].y);                                    \
        }                                                                                                \
        tm_st16(t_src + 16u * (Q), rx);                                                                  \
        tm_st16(t_src + 64u + 16u * (Q), ry);                                                            \
    }
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
// are separate tensor factors.)  Element bits 0..4 run on packed registers:
//   X:  Xa += Xb; Ya += Yb; Xb = Xa - 2 Xb; Yb = Ya - 2 Yb
//   Y:  Xa += Yb; Ya -= Xb; Yb = Xa - 2 Yb; Xb = (-2 Xb) - Ya
// (each one rounding per element, as the scalar forms), element bit 5 on the
// two halves of every register.
// Element bit 5 pairs the halves (a, b) of X[p] and Y[p]; one asm block per
// register pair keeps the halves in their registers (no moves).
__device__ __forceinline__ void k2p_bfly5_x(f2p &X, f2p &Y) {
    asm("{\n\t.reg .f32 ax, bx, ay, by;\n\t"
        "mov.b64 {ax, bx}, %0;\n\tmov.b64 {ay, by}, %1;\n\t"
        "add.rn.f32 ax, ax, bx;\n\tadd.rn.f32 ay, ay, by;\n\t"
        "fma.rn.f32 bx, bx, 0fC0000000, ax;\n\tfma.rn.f32 by, by, 0fC0000000, ay;\n\t"
        "mov.b64 %0, {ax, bx};\n\tmov.b64 %1, {ay, by};\n\t}"
        : "+l"(X), "+l"(Y));
}
__device__ __forceinline__ void k2p_bfly5_y(f2p &X, f2p &Y) {
    asm("{\n\t.reg .f32 ax, bx, ay, by, nay;\n\t"
        "mov.b64 {ax, bx}, %0;\n\tmov.b64 {ay, by}, %1;\n\t"
        "add.rn.f32 ax, ax, by;\n\tsub.rn.f32 ay, ay, bx;\n\t"
        "neg.f32 nay, ay;\n\t"
        "fma.rn.f32 bx, bx, 0fC0000000, nay;\n\tfma.rn.f32 by, by, 0fC0000000, ax;\n\t"
        "mov.b64 %0, {ax, bx};\n\tmov.b64 %1, {ay, by};\n\t}"
        : "+l"(X), "+l"(Y));
}
__device__ __forceinline__ void butterfly_herm_p(f2p (&X)[32], f2p (&Y)[32], uint32_t xyf, uint32_t yf) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        if (!((xyf >> j) & 1u)) continue;
        if ((yf >> j) & 1u) {
#pragma unroll
            for (int p = 0; p < 32; ++p) {
                if ((p >> j) & 1) continue;
                const int q = p | (1 << j);
                X[p] = p_add(X[p], Y[q]);
                Y[p] = p_sub(Y[p], X[q]);
                Y[q] = p_fma(Y[q], kM2, X[p]);
                X[q] = p_sub(p_mul(X[q], kM2), Y[p]);
            }
        } else {
#pragma unroll
            for (int p = 0; p < 32; ++p) {
                if ((p >> j) & 1) continue;
                const int q = p | (1 << j);
                X[p] = p_add(X[p], X[q]);
                Y[p] = p_add(Y[p], Y[q]);
                X[q] = p_fma(X[q], kM2, X[p]);
                Y[q] = p_fma(Y[q], kM2, Y[p]);
            }
        }
    }
    if ((xyf >> 5) & 1u) {
        if ((yf >> 5) & 1u) {
#pragma unroll
            for (int p = 0; p < 32; ++p) k2p_bfly5_y(X[p], Y[p]);
        } else {
#pragma unroll
            for (int p = 0; p < 32; ++p) k2p_bfly5_x(X[p], Y[p]);
        }
    }
}

// Exchanges.  Round A -> B: thread t writes element i (= hi) of its column
// col(lo(t)) in both planes; round B reads its row hi as float4s.  B -> A is
// the reverse.  A thread's round-A addresses are the same in both directions,
// and so are its round-B addresses.
__device__ __forceinline__ void k2p_st2(uint32_t addr_lo, uint32_t addr_hi, f2p v) {
    asm volatile("{\n\t.reg .b32 a, b;\n\tmov.b64 {a, b}, %2;\n\tst.shared.b32 [%0], a;\n\tst.shared.b32 [%1], b;\n\t}" ::"r"(addr_lo),
                 "r"(addr_hi), "l"(v)
                 : "memory");
}
__device__ __forceinline__ f2p k2p_ld2(uint32_t addr_lo, uint32_t addr_hi) {
    f2p v;
    asm volatile("{\n\t.reg .b32 a, b;\n\tld.shared.b32 a, [%1];\n\tld.shared.b32 b, [%2];\n\tmov.b64 %0, {a, b};\n\t}"
                 : "=l"(v)
                 : "r"(addr_lo), "r"(addr_hi)
                 : "memory");
    return v;
}
__device__ __forceinline__ void k2p_st4(uint32_t addr, f2p a, f2p b) {
    asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void k2p_ld4(uint32_t addr, f2p &a, f2p &b) {
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr) : "memory");
}
__device__ __forceinline__ void k2p_store_A(const f2p (&X)[32], const f2p (&Y)[32], float *wk, uint32_t colA) {
    const uint32_t bx = smem_u32(wk + colA), by = bx + 4u * k2pPlane;
#pragma unroll
    for (int p = 0; p < 32; ++p) {
        k2p_st2(bx + 4u * k2pPR * p, bx + 4u * k2pPR * (p + 32), X[p]);
        k2p_st2(by + 4u * k2pPR * p, by + 4u * k2pPR * (p + 32), Y[p]);
    }
}
__device__ __forceinline__ void k2p_load_A(f2p (&X)[32], f2p (&Y)[32], const float *wk, uint32_t colA) {
    const uint32_t bx = smem_u32(wk + colA), by = bx + 4u * k2pPlane;
#pragma unroll
    for (int p = 0; p < 32; ++p) {
        X[p] = k2p_ld2(bx + 4u * k2pPR * p, bx + 4u * k2pPR * (p + 32));
        Y[p] = k2p_ld2(by + 4u * k2pPR * p, by + 4u * k2pPR * (p + 32));
    }
}
__device__ __forceinline__ void k2p_store_B(const f2p (&X)[32], const f2p (&Y)[32], float *wk, uint32_t hi) {
    const uint32_t bx = smem_u32(wk + k2pPR * hi), by = bx + 4u * k2pPlane;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        k2p_st4(bx + 16u * m, X[2 * m], X[2 * m + 1]);
        k2p_st4(by + 16u * m, Y[2 * m], Y[2 * m + 1]);
    }
}
__device__ __forceinline__ void k2p_load_B(f2p (&X)[32], f2p (&Y)[32], const float *wk, uint32_t hi) {
    const uint32_t bx = smem_u32(wk + k2pPR * hi), by = bx + 4u * k2pPlane;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        k2p_ld4(bx + 16u * m, X[2 * m], X[2 * m + 1]);
        k2p_ld4(by + 16u * m, Y[2 * m], Y[2 * m + 1]);
    }
}

// Chunks of C = 10, 11 qubits (TA = C - 6 thread bits per atom, element i of
// thread t at u = t + 2^TA i): atom a of the CTA keeps its planes' rows at
// floats (a / 2^(6-TA)) k2pBuf + (a mod 2^(6-TA)) 68 2^TA (the imaginary plane
// k2pPlane further, as for TA = 6), so the round-B row accesses, the scatter
// positions k2p_pos(u) and the plane offset are unchanged.  Round A: element
// i at row (2^TA i) / 64, column 2 t + c(i), c(i) = 2 ((2^TA i) mod 32) +
// ((2^TA i) mod 64) / 32, a compile-time offset from 8 t.
template <int TA>
__host__ __device__ constexpr int k2p_atom_off(int ai) {
    return (ai >> (6 - TA)) * k2pBuf + (ai & ((1 << (6 - TA)) - 1)) * (k2pPR << TA);
}
template <int TA>
__host__ __device__ constexpr uint32_t k2p_offA(int e) {
    return 4u * (uint32_t)(k2pPR * ((e << TA) >> 6) + 2 * ((e << TA) & 31) + (((e << TA) & 63) >> 5));
}
template <int TA>
__device__ __forceinline__ void k2p_store_A_g(const f2p (&X)[32], const f2p (&Y)[32], float *wk, uint32_t t) {
    const uint32_t bx = smem_u32(wk) + 8u * t, by = bx + 4u * k2pPlane;
#pragma unroll
    for (int p = 0; p < 32; ++p) {
        k2p_st2(bx + k2p_offA<TA>(p), bx + k2p_offA<TA>(p + 32), X[p]);
        k2p_st2(by + k2p_offA<TA>(p), by + k2p_offA<TA>(p + 32), Y[p]);
    }
}
template <int TA>
__device__ __forceinline__ void k2p_load_A_g(f2p (&X)[32], f2p (&Y)[32], const float *wk, uint32_t t) {
    const uint32_t bx = smem_u32(wk) + 8u * t, by = bx + 4u * k2pPlane;
#pragma unroll
    for (int p = 0; p < 32; ++p) {
        X[p] = k2p_ld2(bx + k2p_offA<TA>(p), bx + k2p_offA<TA>(p + 32));
        Y[p] = k2p_ld2(by + k2p_offA<TA>(p), by + k2p_offA<TA>(p + 32));
    }
}
// Round A's elements, each position cleared behind its read.
template <int TA>
__device__ __forceinline__ void k2p_load_A_clear_g(f2p (&X)[32], f2p (&Y)[32], float *wk, uint32_t t) {
    const uint32_t bx = smem_u32(wk) + 8u * t, by = bx + 4u * k2pPlane;
#pragma unroll
    for (int p = 0; p < 32; ++p) {
        X[p] = k2p_ld2(bx + k2p_offA<TA>(p), bx + k2p_offA<TA>(p + 32));
        Y[p] = k2p_ld2(by + k2p_offA<TA>(p), by + k2p_offA<TA>(p + 32));
        k2p_st2(bx + k2p_offA<TA>(p), bx + k2p_offA<TA>(p + 32), 0ull);
        k2p_st2(by + k2p_offA<TA>(p), by + k2p_offA<TA>(p + 32), 0ull);
    }
}
// the last atom's imaginary rows end where the two 64-row atom buffers end
template <int TA>
__host__ __device__ constexpr bool k2p_atoms_tile() {
    return k2p_atom_off<TA>((k2T >> TA) - 1) + k2pPlane + (k2pPR << TA) == 2 * k2pBuf &&
           (k2pPR << TA) * (1 << (6 - TA)) == k2pPlane;
}
static_assert(k2p_atoms_tile<6>() && k2p_atoms_tile<5>() && k2p_atoms_tile<4>(), "atom planes tile the buffers");

// Adjoint CTA = (bin, high pattern f, atom pair kp).  Per setting: round A,
// exchange, round B, the c multiply, inverse round B, exchange, inverse round
// A, and z += v in TMEM (round A's layout).  Two block barriers per setting,
// one in each exchange; they also order the dense c buffers:
//   * setting si reads c buffer si mod 2 between its two barriers;
//   * after the second barrier a thread clears the entries of setting si it
//     scattered itself, then scatters setting si + 1 into the other buffer,
//     whose entries of setting si - 1 were cleared before this setting's
//     first barrier, and which setting si + 1 reads after its first barrier.
// A thread's round-A (round-B) exchange addresses are the same in both
// directions, so it only overwrites addresses that it has read itself.
// C < 12: 2^(13-C) atoms per CTA (round A's layout and the atoms' plane
// offsets as in the cached adjoint below); the dense c buffers are shared by
// all of them, as by the two atoms of C = 12.
template <int C = 12>
__device__ __forceinline__ void adjoint_2r_body(const AdjArgs a, const int cta) {
    if (a.skip && *a.skip) return;
    constexpr int TA = C - 6, APC = k2T >> TA;
    constexpr K2Smem sp = k2p_smem();
    extern __shared__ __align__(16) unsigned char smem[];
    float *cbuf = reinterpret_cast<float *>(smem + sp.fbuf);
    uint32_t *stage_u = reinterpret_cast<uint32_t *>(smem + sp.stage);
    float *stage_c = reinterpret_cast<float *>(smem + sp.stage + 2 * k2Stage * 4);
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
    if (bin >= *a.n_bins) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    const int k = APC * kp + (int)half;
    const bool active = k < a.K;
    float *wk = reinterpret_cast<float *>(smem + sp.work) + k2p_atom_off<TA>((int)half);
    const uint32_t lo = TA == 6 ? k2p_lo(t) : t, colA = k2p_col(lo);
    constexpr uint32_t cmask = (1u << C) - 1u;
    if (warp == 0) tm_alloc(tmem_sm, k2ColsAdj);
    for (int u = tid; u < 2 * k2pPlane; u += k2T) cbuf[u] = 0.f;
    fx_stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, masks_sm, meta_sm);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t t_src = tmem_sm[0] + ((warp * 32u) << 16);
    const uint32_t t_z = t_src + 128u;
    const int bcount = b.count;
    const uint32_t *outcome = a.outcome;
    const float *c_obs = a.c_obs;
    auto issue = [=](int si) {
        if (si < bcount) {
            const SetMeta mt = meta_sm[si];
            const int nst = mt.cnt < k2Stage ? mt.cnt : k2Stage;
            uint32_t *du = stage_u + (si & 1) * k2Stage;
            float *dc = stage_c + (si & 1) * k2Stage;
            for (int j = tid; j < nst; j += k2T) {
                cp_async4(du + j, outcome + mt.lo + j);
                cp_async4(dc + j, c_obs + mt.lo + j);
            }
        }
        cp_async_commit();
    };
    // scatter c 2^-m of setting si into c buffer si mod 2, or clear those
    // entries; each thread touches the entries it staged itself
    auto scatter = [=](int si, bool clear) {
        const SetMeta mt = meta_sm[si];
        const uint32_t *su = stage_u + (si & 1) * k2Stage;
        const float *sc = stage_c + (si & 1) * k2Stage;
        float *cb = cbuf + (si & 1) * k2pPlane;
        for (int j = tid; j < mt.cnt; j += k2T) {
            const bool st = j < k2Stage;
            const uint32_t u = (st ? su[j] : outcome[mt.lo + j]) & cmask;
            cb[k2p_pos(u)] = clear ? 0.f : (st ? sc[j] : c_obs[mt.lo + j]) * mt.cs;
        }
    };
    issue(0);
    k2p_build_source<C>(t_src, a.psi + (size_t)bin * a.src_bin_stride + (size_t)(active ? k : 0) * D, active, f,
                        b.xytop, b.ytop, lo);
    {
        const uint32_t zero[32] = {};
        tm_st(t_z, zero);
        tm_st(t_z + 32u, zero);
        tm_st(t_z + 64u, zero);
        tm_st(t_z + 96u, zero);
    }
    tm_wait_st();
    cp_async_wait0();
    if (bcount > 0) scatter(0, false);  // the c buffers were zeroed before the barrier above
    issue(1);
    f2p X[32], Y[32];
    for (int si = 0; si < bcount; ++si) {
        const uint2 mk = masks_sm[si];
        k2p_tm_ld(t_src, X, Y);
        // the four rounds (A, B, then B, A conjugate-transposed = the same
        // Hermitian factors) share one butterfly site; between them: the
        // exchange A -> B, the c multiply, the exchange B -> A
#pragma unroll 1
        for (int ph = 0; ph < 4; ++ph) {
            const bool rA = ph == 0 || ph == 3;  // round A: chunk bits 6..C-1, round B: bits 0..5
            const uint32_t sh = rA ? (uint32_t)TA : 0u, keep = rA ? 63u & ~((1u << (6 - TA)) - 1u) : 63u;
            butterfly_herm_p(X, Y, (mk.x >> sh) & keep, (mk.y >> sh) & keep);
            if (ph == 0) {
                if constexpr (TA == 6) k2p_store_A(X, Y, wk, colA);
                else k2p_store_A_g<TA>(X, Y, wk, t);
                __syncthreads();
                k2p_load_B(X, Y, wk, t);
            } else if (ph == 1) {
                const uint32_t crow = smem_u32(cbuf + (si & 1) * k2pPlane + k2pPR * t);
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    f2p c0, c1;
                    k2p_ld4(crow + 16u * m, c0, c1);
                    X[2 * m] = p_mul(X[2 * m], c0);
                    Y[2 * m] = p_mul(Y[2 * m], c0);
                    X[2 * m + 1] = p_mul(X[2 * m + 1], c1);
                    Y[2 * m + 1] = p_mul(Y[2 * m + 1], c1);
                }
            } else if (ph == 2) {
                k2p_store_B(X, Y, wk, t);
                __syncthreads();
                if constexpr (TA == 6) k2p_load_A(X, Y, wk, colA);
                else k2p_load_A_g<TA>(X, Y, wk, t);
            }
        }
        k2p_tm_acc(t_z, X, Y);
        scatter(si, true);
        cp_async_wait0();
        if (si + 1 < bcount) scatter(si + 1, false);
        issue(si + 2);
    }
    cp_async_wait0();
    tm_wait_st();
    k2p_tm_ld(t_z, X, Y);  // every warp whole (.sync.aligned: 16-thread atoms share warps)
    if (active) {
        float2 *zo = a.zbuf + ((size_t)bin * a.K + k) * D + ((size_t)f << C) + lo;
#pragma unroll
        for (int p = 0; p < 32; ++p) {
            float xa, xb, ya, yb;
            p_unpack(X[p], xa, xb);
            p_unpack(Y[p], ya, yb);
            zo[(uint32_t)p << TA] = make_float2(xa, ya);
            zo[(uint32_t)(p + 32) << TA] = make_float2(xb, yb);
        }
    }
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(tmem_sm[0], k2ColsAdj);
    }
}
template <int C = 12>
__global__ void __launch_bounds__(k2T, 2) k_adjoint_2r(const AdjArgs a) {
    adjoint_2r_body<C>(a, blockIdx.x);
}
template <int C = 12>
__global__ void __launch_bounds__(k2T, 2) k_adjoint_2r_multi(const AdjArgs *__restrict__ args, const int *__restrict__ start, int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const AdjArgs a = args[i];
    adjoint_2r_body<C>(a, (int)blockIdx.x - start[i]);
}

// Cached adjoint (the evaluate path): the forward kernel has stored the chunk
// transform phi = K_s psi_k of every setting at its observed outcomes (K_s the
// unscaled chunk transform, a.phi_obs), so y = c 2^-m phi is known without
// recomputing the forward rounds, and only the inverse rounds run:
//   z += K_s^* y = (round A)(round B) y  for every setting of the bin.
// CTA = (bin, high pattern f, atom pair kp) as in k_adjoint_2r, but the two
// atoms' 64-thread halves never wait on each other: each stages its own
// (outcome, c, phi) entries with cp.async (double-buffered), so every barrier
// inside the setting loop is an atom barrier.  Per setting and atom:
//   scatter y into the (zeroed) exchange planes at the observed positions;
//   barrier; load round B's row; inverse round B; store the row back;
//   barrier; load round A's column, zero those positions; inverse round A;
//   z += v (TMEM); barrier (the zeroing is done before the next scatter).
// A thread scatters and stages the same entries (j = t, t + 64, ...), so its
// own cp.async wait makes them visible to it, and the staging buffer it
// refills for setting si + 1 was last read by itself (setting si - 1).
// How many entries per setting are staged (the scatter reads the rest from
// global memory) trades latency against occupancy:
//   * k_adjoint_2c stages none in shared memory: each thread loads its first
//     two entries of the next setting into registers at the end of the current
//     one.  A CTA takes 71,952 B and, with at most 168 registers a thread,
//     three CTAs (12 warps) share an SM.  The n = 16, M = 4096, K = 16 launch
//     (about 120 entries per setting and chunk) takes 5.54 ms, against 5.63
//     with 32 entries staged by cp.async and 5.82 with 512 at two CTAs per SM;
//   * k_adjoint_2c_multi (the batch, whose settings hold up to 5000 entries
//     per chunk) stages 512 at two CTAs per SM: 4.79 against 5.16 ms with 32.
constexpr int k2cStageSingle = 0;   // observed entries per setting and atom staged by cp.async
constexpr int k2cStageMulti = 512;
struct K2cSmem {
    int work, stage_u, stage_c, stage_p, masks, meta, tmem, total;
};
__host__ __device__ constexpr K2cSmem k2c_smem(int k2cStage) {
    K2cSmem sp{};
    sp.work = 0;
    sp.stage_p = sp.work + 2 * k2pBuf * 4;                 // [atom][buffer][entry] float2
    sp.stage_u = sp.stage_p + 2 * 2 * k2cStage * 8;        // [atom][buffer][entry] uint32
    sp.stage_c = sp.stage_u + 2 * 2 * k2cStage * 4;        // [atom][buffer][entry] float
    sp.masks = sp.stage_c + 2 * 2 * k2cStage * 4;
    sp.meta = sp.masks + kMaxBin * (int)sizeof(uint2);
    sp.tmem = sp.meta + kMaxBin * (int)sizeof(SetMeta);
    sp.total = sp.tmem + 16;
    return sp;
}
__host__ __device__ constexpr bool k2c_aligned(int st) {
    return k2c_smem(st).stage_p % 16 == 0 && k2c_smem(st).stage_u % 16 == 0 && k2c_smem(st).stage_c % 16 == 0 &&
           k2c_smem(st).masks % 16 == 0 && k2c_smem(st).meta % 16 == 0;
}
static_assert(k2c_aligned(k2cStageSingle) && k2c_aligned(k2cStageMulti), "aligned shared arrays");
constexpr uint32_t k2cCols = 128;  // TMEM columns of a cached-adjoint CTA: the accumulator
constexpr int k2cCta = k2c_smem(k2cStageSingle).total + 1024;
constexpr int k2cCtaMulti = k2c_smem(k2cStageMulti).total + 1024;
// Every mix of two-round forward, adjoint and cached-adjoint CTAs that shared
// memory admits on one SM fits in its 512 TMEM columns, so an allocation never
// waits (CTAs of different kernels share an SM when the batched graph runs
// instances concurrently).
__host__ __device__ constexpr bool k2_tmem_fits() {
    for (int na = 0; na <= 4; ++na)
        for (int nc = 0; nc <= 4; ++nc)
            for (int nm = 0; nm <= 4; ++nm)
                for (int nf = 0; nf <= 4; ++nf)
                    if (na * k2CtaAdj + nc * k2cCta + nm * k2cCtaMulti + nf * k2CtaFwd <= k2SmemSM &&
                        na * (int)k2ColsAdj + (nc + nm) * (int)k2cCols + nf * (int)k2ColsFwd > 512)
                        return false;
    return true;
}
static_assert(3 * k2cCta <= k2SmemSM && 4 * k2cCta > k2SmemSM && 2 * k2cCtaMulti <= k2SmemSM &&
                  3 * k2cCtaMulti > k2SmemSM && k2_tmem_fits(),
              "cached-adjoint occupancy and TMEM");

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

// C < 12: 2^(13-C) atoms per CTA; each stages 2 k2cStage / 2^(13-C)
// entries per setting (the same shared memory in all).
template <int k2cStage, int C = 12>
__device__ __forceinline__ void adjoint_2c_body(const AdjArgs a, const int cta) {
    if (a.skip && *a.skip) return;
    constexpr int TA = C - 6, APC = k2T >> TA, SA = 2 * k2cStage / APC;  // per-atom staged entries
    constexpr K2cSmem sp = k2c_smem(k2cStage);
    extern __shared__ __align__(16) unsigned char smem[];
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
    if (bin >= *a.n_bins) return;
    const Bin b = a.bins[bin];
    const int D = 1 << a.n;
    const int k = APC * kp + (int)half;
    const bool active = k < a.K;
    float *wk = reinterpret_cast<float *>(smem + sp.work) + k2p_atom_off<TA>((int)half);
    float2 *stp = reinterpret_cast<float2 *>(smem + sp.stage_p) + half * 2 * SA;
    uint32_t *stu = reinterpret_cast<uint32_t *>(smem + sp.stage_u) + half * 2 * SA;
    float *stc = reinterpret_cast<float *>(smem + sp.stage_c) + half * 2 * SA;
    // round A: TA = 6 permutes the columns among the threads (conflict-free stores)
    const uint32_t lo = TA == 6 ? k2p_lo(t) : t, colA = k2p_col(lo);
    constexpr uint32_t cmask = (1u << C) - 1u;
    if (warp == 0) tm_alloc(tmem_sm, k2cCols);
    for (int u = tid; u < 2 * k2pBuf; u += k2T) reinterpret_cast<float *>(smem + sp.work)[u] = 0.f;
    fx_stage_bin(b, f, (1 << a.r) + 1, a.order, a.plans, a.row_ptr, a.choff, masks_sm, meta_sm);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t t_z = tmem_sm[0] + ((warp * 32u) << 16);
    const int bcount = b.count;
    const uint32_t *outcome = a.outcome;
    const float *c_obs = a.c_obs;
    const float2 *phk = a.phi_obs + (size_t)(active ? k : 0) * a.nnz;
    {
        const f2p zero[16] = {};
#pragma unroll
        for (int q = 0; q < 4; ++q) k2p_tm_st16(t_z + 32u * q, zero);
    }
    f2p X[32], Y[32];
    // The TMEM accesses (.sync.aligned) need whole warps: atoms of 16 threads
    // share a warp, so there an inactive atom (k >= K) runs the loop too, on
    // atom 0's entries in its own planes (cleared behind every setting), and
    // only its z write is skipped.  Larger atoms are whole warps.
    const bool run = TA >= 5 ? active : true;
    if (run) {
        // k2cStage == 0: each thread loads its first two entries of the next
        // setting into registers at the end of the current one (X, Y are dead
        // there, so the loads cost no registers at the kernel's peak) and finds
        // them in flight-completed registers at the next scatter.
        uint32_t ru[2] = {0u, 0u};
        float rc[2] = {0.f, 0.f};
        float2 rp[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        auto prefetch = [&](int si) {
            if (si < bcount) {
                const SetMeta mt = meta_sm[si];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int j = (int)t + (e << TA);
                    if (j < mt.cnt) {
                        ru[e] = outcome[mt.lo + j];
                        rc[e] = c_obs[mt.lo + j];
                        rp[e] = phk[mt.lo + j];
                    }
                }
            }
        };
        auto issue = [&](int si) {
            if constexpr (k2cStage == 0) return;
            if (si < bcount) {
                const SetMeta mt = meta_sm[si];
                const int nst = mt.cnt < SA ? mt.cnt : SA;
                const int o = (si & 1) * SA;
                for (int j = t; j < nst; j += (1 << TA)) {
                    cp_async4(stu + o + j, outcome + mt.lo + j);
                    cp_async4(stc + o + j, c_obs + mt.lo + j);
                    cp_async8(stp + o + j, phk + mt.lo + j);
                }
            }
            cp_async_commit();
        };
        if constexpr (k2cStage == 0) prefetch(0);
        else issue(0);
        for (int si = 0; si < bcount; ++si) {
            const uint2 mk = masks_sm[si];
            const SetMeta mt = meta_sm[si];
            if constexpr (k2cStage == 0) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int j = (int)t + (e << TA);
                    if (j < mt.cnt) {
                        const uint32_t pos = k2p_pos(ru[e] & cmask);
                        const float cy = rc[e] * mt.cs;
                        wk[pos] = cy * rp[e].x;
                        wk[k2pPlane + pos] = cy * rp[e].y;
                    }
                }
                for (int j = (int)t + (2 << TA); j < mt.cnt; j += (1 << TA)) {
                    const uint32_t pos = k2p_pos(outcome[mt.lo + j] & cmask);
                    const float cy = c_obs[mt.lo + j] * mt.cs;
                    const float2 ph = phk[mt.lo + j];
                    wk[pos] = cy * ph.x;
                    wk[k2pPlane + pos] = cy * ph.y;
                }
            } else {
                cp_async_wait0();  // this thread's entries of setting si have landed
                issue(si + 1);     // into the buffer this thread read for setting si - 1
                const int o = (si & 1) * SA;
                for (int j = t; j < mt.cnt; j += (1 << TA)) {
                    const bool st = j < SA;
                    const uint32_t u = (st ? stu[o + j] : outcome[mt.lo + j]) & cmask;
                    const float cy = (st ? stc[o + j] : c_obs[mt.lo + j]) * mt.cs;
                    const float2 ph = st ? stp[o + j] : phk[mt.lo + j];
                    const uint32_t pos = k2p_pos(u);
                    wk[pos] = cy * ph.x;
                    wk[k2pPlane + pos] = cy * ph.y;
                }
            }
            k2_bar_atom_g<TA>(half);  // the scatter is visible
            k2p_load_B(X, Y, wk, t);
            // the inverse rounds (the Hermitian chunk factors are their own
            // conjugate transposes): round B, then round A
#pragma unroll 1
            for (int ph = 0; ph < 2; ++ph) {
                const uint32_t sh = ph ? (uint32_t)TA : 0u, keep = ph ? 63u & ~((1u << (6 - TA)) - 1u) : 63u;
                butterfly_herm_p(X, Y, (mk.x >> sh) & keep, (mk.y >> sh) & keep);
                if (ph == 0) {
                    k2p_store_B(X, Y, wk, t);
                    k2_bar_atom_g<TA>(half);
                    if constexpr (TA == 6) {
                        k2p_load_A(X, Y, wk, colA);
                        const uint32_t bx = smem_u32(wk + colA), by = bx + 4u * k2pPlane;
#pragma unroll
                        for (int p = 0; p < 32; ++p) {
                            k2p_st2(bx + 4u * k2pPR * p, bx + 4u * k2pPR * (p + 32), 0ull);
                            k2p_st2(by + 4u * k2pPR * p, by + 4u * k2pPR * (p + 32), 0ull);
                        }
                    } else {
                        k2p_load_A_clear_g<TA>(X, Y, wk, t);
                    }
                }
            }
            k2p_tm_acc(t_z, X, Y);
            if constexpr (k2cStage == 0) prefetch(si + 1);
            k2_bar_atom_g<TA>(half);  // every position is zero again before the next scatter
        }
        cp_async_wait0();
    }
    tm_wait_st();
    if (run) k2p_tm_ld(t_z, X, Y);
    if (active) {
        float2 *zo = a.zbuf + ((size_t)bin * a.K + k) * D + ((size_t)f << C) + lo;
#pragma unroll
        for (int p = 0; p < 32; ++p) {
            float xa, xb, ya, yb;
            p_unpack(X[p], xa, xb);
            p_unpack(Y[p], ya, yb);
            zo[(uint32_t)p << TA] = make_float2(xa, ya);
            zo[(uint32_t)(p + 32) << TA] = make_float2(xb, yb);
        }
    }
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(tmem_sm[0], k2cCols);
    }
}
template <int C = 12>
__global__ void __launch_bounds__(k2T, 3) k_adjoint_2c(const AdjArgs a) {
    adjoint_2c_body<k2cStageSingle, C>(a, blockIdx.x);
}
template <int C = 12>
__global__ void __launch_bounds__(k2T, 2) k_adjoint_2c_multi(const AdjArgs *__restrict__ args, const int *__restrict__ start, int count) {
    const int i = multi_find(start, count, (int)blockIdx.x);
    const AdjArgs a = args[i];
    adjoint_2c_body<k2cStageMulti, C>(a, (int)blockIdx.x - start[i]);
}
