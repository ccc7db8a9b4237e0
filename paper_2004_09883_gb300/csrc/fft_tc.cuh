// fft_tc.cuh -- radix-16 Stockham stages on the tensor cores (tcgen05).
//
// A radix-16 stage applies the 16-point DFT matrix W[j][r] = exp(s 2 pi i j r / 16)
// to the (twiddled) 16 inputs of every butterfly.  Written over reals, one
// butterfly is a row vector times a 32 x 32 matrix:
//     [yr | yi] = [xr | xi] * M,   M = [[Wr^T, Wi^T], [-Wi^T, Wr^T]],
// so a stage over 128 butterflies is one (128 x 32) x (32 x 32) product.  The
// tensor cores take FP16 operands, so every value is split in two halves,
// x = x_hi + x_lo with x_hi = fp16(x) and x_lo = fp16(x - x_hi) (and M the
// same way); the three products x_hi M_hi + x_lo M_hi + x_hi M_lo are summed in
// an FP32 accumulator (the x_lo M_lo term, ~2^-22 relative, is dropped).  Before
// the split each butterfly's inputs are scaled by a power of two that brings
// its largest component into [0.5, 1), and its outputs are scaled back (both
// exact), so the FP16 range never clips and the split keeps ~22 bits.
//
// Mapping onto tcgen05 (cta_group::1, kind::f16, M = 128, N = 32, K = 16 per
// instruction): thread i of a 128-thread group owns butterfly row i; it writes
// its row of A = [x_hi (32 halves) | x_lo (32 halves)] into shared memory in the
// K-major no-swizzle layout (8 x 16-byte core matrices: 128 bytes between
// K-neighbours, 1024 bytes between 8-row groups); B^T = [M_hi | M_lo] (32 rows
// x 64 halves) is built once per CTA in the same layout.  One thread issues 6
// MMAs per group into TMEM columns [32 g, 32 g + 32) and commits them to an
// mbarrier; every thread then reads its accumulator row (tcgen05.ld 32x32b,
// warp w reads lanes 32 (w % 4) ...) and scatters the 16 outputs.
#pragma once

#include <cuda_fp16.h>

#include "fft_device.cuh"

namespace fbfft {

constexpr int kTcRowBytes = 128;                 // one A row: 64 halves
constexpr int kTcGroupBytes = 128 * kTcRowBytes; // one 128-row A tile
constexpr int kTcBBytes = 32 * 128;              // B^T: 32 rows x 64 halves
constexpr int kTcLbo = 128;                      // bytes between K-adjacent core matrices
constexpr int kTcSbo = 1024;                     // bytes between 8-row groups (8 core matrices per row group)

// Where the A rows live: TMEM (default; written with tcgen05.st, read by the
// MMA as its A operand) or shared memory (FB_FFT_TC_A_SMEM; the work buffer,
// through a K-major descriptor).
#ifdef FB_FFT_TC_A_SMEM
constexpr bool kTcATmem = false;
#else
constexpr bool kTcATmem = true;
#endif

// TMEM columns a CTA of `threads` compute threads allocates: 32 accumulator
// columns per 128-row group, and as many again for the A rows when they live
// in TMEM (power of two >= 32).
__host__ __device__ constexpr int tc_tmem_cols(int threads)
{
    return (threads / 128) * 32 * (kTcATmem ? 2 : 1) < 32 ? 32 : (threads / 128) * 32 * (kTcATmem ? 2 : 1);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading- and
// stride-dimension byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr)
{
    unsigned long long d = (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)((kTcLbo >> 4) & 0x3FFF) << 16;
    d |= (unsigned long long)((kTcSbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    return d;
}
// Instruction descriptor, kind::f16: FP32 accumulator, FP16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr unsigned tc_idesc(int M, int N)
{
    return (1u << 4) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

// The column count is an immediate, so the toolchain sees how much TMEM a CTA takes.
template <int NCOLS>
__device__ __forceinline__ void tc_alloc(unsigned* slot)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "n"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int NCOLS>
__device__ __forceinline__ void tc_dealloc(unsigned taddr)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NCOLS) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_mma(unsigned dt, unsigned long long ad, unsigned long long bd, unsigned idesc,
                                       unsigned accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Arrive once on `bar` when every MMA this thread issued before has completed.
__device__ __forceinline__ void tc_commit(unsigned long long* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// A operand from TMEM: [a-tmem] instead of a shared-memory descriptor.
__device__ __forceinline__ void tc_mma_ta(unsigned dt, unsigned at, unsigned long long bd, unsigned idesc,
                                          unsigned accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(dt),
        "r"(at), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane, then wait for them.
__device__ __forceinline__ void tc_st16(unsigned taddr, const unsigned (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(unsigned taddr, unsigned (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void st_shared_v4(unsigned addr, unsigned a, unsigned b, unsigned c, unsigned d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// B^T = [M_hi | M_lo] for direction FWD, in the K-major layout (all compute threads).
template <int THREADS, bool FWD>
__device__ __forceinline__ void tc_build_b(unsigned char* b)
{
    for (int e = threadIdx.x; e < 32 * 64; e += THREADS) {
        const int n = e >> 6, k = e & 63;
        const int kk = k & 31;
        const int r = kk & 15, jj = n & 15;
        float s, c;
        // FP32 is enough: the FP16 pair keeps ~22 bits; FP64 is a slow unit on this part
        sincospif((float)((jj * r) & 15) * 0.125f, &s, &c);  // exp(s 2 pi i j r / 16) = c + i (sign) s
        const float wr = c, wi = FWD ? -s : s;
        const float val = kk < 16 ? (n < 16 ? wr : wi) : (n < 16 ? -wi : wr);
        const __half hi = __float2half_rn(val);
        const __half out = k < 32 ? hi : __float2half_rn(val - __half2float(hi));
        const int off = (n >> 3) * kTcSbo + (k >> 3) * kTcLbo + (n & 7) * 16 + (k & 7) * 2;
        *reinterpret_cast<__half*>(b + off) = out;
    }
}

struct TcState {
    unsigned tmem;             // TMEM base address (lane 0, first column): accumulators
    unsigned long long* bar;   // MMA completion mbarrier
    unsigned bsm;              // shared address of B^T
    unsigned uses;             // completed MMA rounds (mbarrier phase)
    unsigned a;                // TMEM address of the A rows (when kTcATmem)
};

// The scale exponent of a butterfly: 2^-e brings its largest component into [0.5, 1).
__device__ __forceinline__ int tc_scale_exp(const float2 (&v)[16])
{
    float m = 0.f;
#pragma unroll
    for (int r = 0; r < 16; ++r) m = fmaxf(m, fmaxf(fabsf(v[r].x), fabsf(v[r].y)));
    const int e = ((__float_as_int(m) >> 23) & 0xff) - 126;  // m in [2^(e-1), 2^e)
    return e < -126 ? -126 : (e > 126 ? 126 : e);
}
// K pair p (K = 2p, 2p+1; 0..15 real parts, 16..31 imaginary parts) of the
// scaled butterfly as packed halves: hi and lo words.
__device__ __forceinline__ void tc_split_pair(const float2 (&v)[16], float down, int p, unsigned& hw, unsigned& lw)
{
    const int k0 = 2 * p;
    const float a = (k0 < 16 ? v[k0].x : v[k0 - 16].y) * down;
    const float b = (k0 + 1 < 16 ? v[k0 + 1].x : v[k0 + 1 - 16].y) * down;
    const __half2 h = __floats2half2_rn(a, b);  // (a, b) -> low, high half
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hw = *reinterpret_cast<const unsigned*>(&h);
    lw = *reinterpret_cast<const unsigned*>(&l);
}

// TMEM variant: scale, split and write this thread's row of A (hi: 16
// columns, lo: the next 16) into its lane; waits for the stores.  Returns e.
__device__ __forceinline__ int tc_put_row_tmem(const float2 (&v)[16], const TcState& tc)
{
    const int e = tc_scale_exp(v);
    const float down = __int_as_float((127 - e) << 23);
    unsigned hw[16], lw[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) tc_split_pair(v, down, p, hw[p], lw[p]);
    const int warp = threadIdx.x >> 5;
    const unsigned row = tc.a + ((unsigned)(32 * (warp & 3)) << 16) + 32u * (unsigned)(warp >> 2);
    tc_st16(row, hw);
    tc_st16(row + 16, lw);
    tc_wait_st();
    return e;
}

// TMEM variant of the issue: A operands [a_g + 0 / 8] (hi, K 0-15 / 16-31) and
// [a_g + 16 / 24] (lo), 8 columns = 16 halves per K step.
template <int GROUPS>
__device__ __forceinline__ void tc_issue_tmem(const TcState& tc)
{
    constexpr unsigned idesc = tc_idesc(128, 32);
    tc_fence_after();
#pragma unroll
    for (int g = 0; g < GROUPS; ++g) {
        const unsigned a = tc.a + 32 * g, d = tc.tmem + 32 * g;
        tc_mma_ta(d, a, tc_desc(tc.bsm), idesc, 0);                                  // hi * M_hi
        tc_mma_ta(d, a + 8, tc_desc(tc.bsm + 2 * kTcLbo), idesc, 1);
        tc_mma_ta(d, a + 16, tc_desc(tc.bsm), idesc, 1);                             // lo * M_hi
        tc_mma_ta(d, a + 24, tc_desc(tc.bsm + 2 * kTcLbo), idesc, 1);
        tc_mma_ta(d, a, tc_desc(tc.bsm + 4 * kTcLbo), idesc, 1);                     // hi * M_lo
        tc_mma_ta(d, a + 8, tc_desc(tc.bsm + 6 * kTcLbo), idesc, 1);
    }
    tc_commit(tc.bar);
}

// Scale, split and store this thread's butterfly as A row `row` of group `grp`
// (A tiles start at shared address `abase`).  Returns the exponent e of the
// scale 2^-e applied.
__device__ __forceinline__ int tc_put_row(const float2 (&v)[16], unsigned abase, int grp, int row)
{
    const int e = tc_scale_exp(v);
    const float down = __int_as_float((127 - e) << 23);
    const unsigned rowaddr = abase + grp * kTcGroupBytes + (row >> 3) * kTcSbo + (row & 7) * 16;
    // chunks 0..3 hi, 4..7 lo (8 halves each)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        unsigned hw[4], lw[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) tc_split_pair(v, down, 4 * c + p, hw[p], lw[p]);
        st_shared_v4(rowaddr + c * kTcLbo, hw[0], hw[1], hw[2], hw[3]);
        st_shared_v4(rowaddr + (4 + c) * kTcLbo, lw[0], lw[1], lw[2], lw[3]);
    }
    return e;
}

// One thread: the 6 MMAs of every group, then the commit.
template <int GROUPS>
__device__ __forceinline__ void tc_issue(const TcState& tc, unsigned abase)
{
    constexpr unsigned idesc = tc_idesc(128, 32);
    tc_fence_after();
#pragma unroll
    for (int g = 0; g < GROUPS; ++g) {
        const unsigned a = abase + g * kTcGroupBytes, d = tc.tmem + 32 * g;
        tc_mma(d, tc_desc(a), tc_desc(tc.bsm), idesc, 0);                                      // hi * M_hi
        tc_mma(d, tc_desc(a + 2 * kTcLbo), tc_desc(tc.bsm + 2 * kTcLbo), idesc, 1);
        tc_mma(d, tc_desc(a + 4 * kTcLbo), tc_desc(tc.bsm), idesc, 1);                         // lo * M_hi
        tc_mma(d, tc_desc(a + 6 * kTcLbo), tc_desc(tc.bsm + 2 * kTcLbo), idesc, 1);
        tc_mma(d, tc_desc(a), tc_desc(tc.bsm + 4 * kTcLbo), idesc, 1);                         // hi * M_lo
        tc_mma(d, tc_desc(a + 2 * kTcLbo), tc_desc(tc.bsm + 6 * kTcLbo), idesc, 1);
    }
    tc_commit(tc.bar);
}

// This thread's 16 outputs from its accumulator row, scaled back by 2^e.
__device__ __forceinline__ void tc_get_row(const TcState& tc, int e, float2 (&y)[16])
{
    const int warp = threadIdx.x >> 5;
    unsigned r[32];
    tc_ld32(tc.tmem + ((unsigned)(32 * (warp & 3)) << 16) + 32u * (unsigned)(warp >> 2), r);
    tc_fence_before();
    const float up = __int_as_float((127 + e) << 23);
#pragma unroll
    for (int i = 0; i < 16; ++i) y[i] = make_float2(__uint_as_float(r[i]) * up, __uint_as_float(r[16 + i]) * up);
}

}  // namespace fbfft
