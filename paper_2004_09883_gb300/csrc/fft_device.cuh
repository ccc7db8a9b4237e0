// fft_device.cuh -- register-level DFT butterflies and the Stockham line pass.
//
// A length-L line is transformed by mixed-radix Stockham autosort stages
// (radices 16, 8, 5, 4, 3, 2).  Stage s with radix R, after Ns = product of
// the earlier radices, takes butterfly j (0 <= j < L/R) with k = j mod Ns:
//   v[r]  = a[j + r*L/R] * w_{Ns*R}^{r*k}          (r = 0..R-1)
//   V     = R-point DFT of v
//   b[(j-k)*R + k + r*Ns] = V[r]
// which after the last stage leaves X[k] in natural order (Stockham's
// self-sorting form of the Cooley-Tukey factorisation).  The first stage reads
// global memory directly and the last writes it directly; stages in between
// exchange through shared memory, so a two-stage line (L <= 256) touches shared
// memory once.
#pragma once

#include <cuda_runtime.h>

#include <cstdio>

#include "fb_internal.h"

namespace fbfft {

// Complex add and subtract.  On sm_100 and later the device path issues one
// paired FP32 instruction (add.rn.f32x2) per complex value, the same two
// round-to-nearest results as two scalar adds with half the issue slots.
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
#else
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
#endif
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }

__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * w for the forward sign, a * conj(w) for the inverse (tables hold exp(-...)).
template <bool FWD>
__host__ __device__ __forceinline__ float2 twmul(float2 a, float2 w)
{
    return FWD ? make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x)
               : make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
// z * (s*i), s = -1 forward, +1 inverse.
template <bool FWD>
__host__ __device__ __forceinline__ float2 mul_si(float2 z)
{
    return FWD ? make_float2(z.y, -z.x) : make_float2(-z.y, z.x);
}
// z * (C + s*i*S)  ==  C*z + S*(s*i*z)
template <bool FWD>
__host__ __device__ __forceinline__ float2 rot(float2 z, float C, float S)
{
    const float2 q = mul_si<FWD>(z);
    return make_float2(C * z.x + S * q.x, C * z.y + S * q.y);
}

// Constants: cos/sin of 2*pi*m/16, 2*pi/3, 2*pi/5, 4*pi/5.
#define FB_C16_1 0.92387953251128675613f  // cos(pi/8)
#define FB_S16_1 0.38268343236508977173f  // sin(pi/8)
#define FB_R2    0.70710678118654752440f  // sqrt(2)/2
#define FB_S3    0.86602540378443864676f  // sin(2pi/3)
#define FB_C5_1  0.30901699437494742410f  // cos(2pi/5)
#define FB_C5_2 -0.80901699437494742410f  // cos(4pi/5)
#define FB_S5_1  0.95105651629515357212f  // sin(2pi/5)
#define FB_S5_2  0.58778525229247312917f  // sin(4pi/5)

template <bool FWD>
__host__ __device__ __forceinline__ void dft2(float2& a, float2& b)
{
    const float2 t = a;
    a = t + b;
    b = t - b;
}

// t +- (s i) d, written per component: the (s i) product swaps d's halves,
// which a paired add could only take after two moves.
template <bool FWD>
__host__ __device__ __forceinline__ void add_sub_si(float2 t, float2 d, float2& plus, float2& minus)
{
    if (FWD) {
        plus = make_float2(t.x + d.y, t.y - d.x);
        minus = make_float2(t.x - d.y, t.y + d.x);
    } else {
        plus = make_float2(t.x - d.y, t.y + d.x);
        minus = make_float2(t.x + d.y, t.y - d.x);
    }
}

template <bool FWD>
__host__ __device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3)
{
    const float2 t0 = v0 + v2, t1 = v0 - v2, t2 = v1 + v3, d = v1 - v3;
    v0 = t0 + t2;
    v2 = t0 - t2;
    add_sub_si<FWD>(t1, d, v1, v3);  // t1 +- (s i) (v1 - v3)
}
// dft4 of (v0, v1, (s i) v2, v3): the third input's factor folded into its adds.
template <bool FWD>
__host__ __device__ __forceinline__ void dft4_si2(float2& v0, float2& v1, float2& v2, float2& v3)
{
    float2 t0, t1;
    add_sub_si<FWD>(v0, v2, t0, t1);
    const float2 t2 = v1 + v3, d = v1 - v3;
    v0 = t0 + t2;
    v2 = t0 - t2;
    add_sub_si<FWD>(t1, d, v1, v3);
}

template <bool FWD>
__host__ __device__ __forceinline__ void dft3(float2& a, float2& b, float2& c)
{
    const float2 t = b + c;
    const float2 m = a - 0.5f * t;
    const float2 d = FB_S3 * mul_si<FWD>(b - c);
    a = a + t;
    b = m + d;
    c = m - d;
}

template <bool FWD>
__host__ __device__ __forceinline__ void dft5(float2* v)
{
    const float2 t1 = v[1] + v[4], t2 = v[2] + v[3], t3 = v[1] - v[4], t4 = v[2] - v[3];
    const float2 a1 = make_float2(v[0].x + FB_C5_1 * t1.x + FB_C5_2 * t2.x, v[0].y + FB_C5_1 * t1.y + FB_C5_2 * t2.y);
    const float2 a2 = make_float2(v[0].x + FB_C5_2 * t1.x + FB_C5_1 * t2.x, v[0].y + FB_C5_2 * t1.y + FB_C5_1 * t2.y);
    const float2 b1 = mul_si<FWD>(make_float2(FB_S5_1 * t3.x + FB_S5_2 * t4.x, FB_S5_1 * t3.y + FB_S5_2 * t4.y));
    const float2 b2 = mul_si<FWD>(make_float2(FB_S5_2 * t3.x - FB_S5_1 * t4.x, FB_S5_2 * t3.y - FB_S5_1 * t4.y));
    v[0] = v[0] + t1 + t2;
    v[1] = a1 + b1;
    v[4] = a1 - b1;
    v[2] = a2 + b2;
    v[3] = a2 - b2;
}

// 8 = 2 x 4: even/odd 4-point DFTs, then Y[k] = E[k] +- w8^k O[k].
template <bool FWD>
__host__ __device__ __forceinline__ void dft8(float2* v)
{
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<FWD>(e0, e1, e2, e3);
    dft4<FWD>(o0, o1, o2, o3);
    o1 = rot<FWD>(o1, FB_R2, FB_R2);
    o3 = rot<FWD>(o3, -FB_R2, FB_R2);
    v[0] = e0 + o0;
    v[4] = e0 - o0;
    v[1] = e1 + o1;
    v[5] = e1 - o1;
    add_sub_si<FWD>(e2, o2, v[2], v[6]);  // e2 +- w8^2 o2, w8^2 = s i
    v[3] = e3 + o3;
    v[7] = e3 - o3;
}

// 16 = 4 x 4: with r = 4*r1 + r2 and k = k1 + 4*k2,
// w16^{rk} = w4^{r1 k1} w16^{r2 k1} w4^{r2 k2}.
template <bool FWD>
__host__ __device__ __forceinline__ void dft16(float2* v)
{
#pragma unroll
    for (int r2 = 0; r2 < 4; ++r2) dft4<FWD>(v[r2], v[4 + r2], v[8 + r2], v[12 + r2]);
    // v[4*k1 + r2] now holds A[r2][k1]; multiply by w16^{r2*k1}
    v[5] = rot<FWD>(v[5], FB_C16_1, FB_S16_1);    // (1,1): m=1
    v[6] = rot<FWD>(v[6], FB_R2, FB_R2);          // k1=1, r2=2: m=2
    v[7] = rot<FWD>(v[7], FB_S16_1, FB_C16_1);    // k1=1, r2=3: m=3
    v[9] = rot<FWD>(v[9], FB_R2, FB_R2);          // k1=2, r2=1: m=2
    // k1=2, r2=2: m=4, w16^4 = s i, folded into the row's dft4 below
    v[11] = rot<FWD>(v[11], -FB_R2, FB_R2);       // k1=2, r2=3: m=6
    v[13] = rot<FWD>(v[13], FB_S16_1, FB_C16_1);  // k1=3, r2=1: m=3
    v[14] = rot<FWD>(v[14], -FB_R2, FB_R2);       // k1=3, r2=2: m=6
    v[15] = rot<FWD>(v[15], -FB_C16_1, -FB_S16_1);// k1=3, r2=3: m=9
    dft4<FWD>(v[0], v[1], v[2], v[3]);
    dft4<FWD>(v[4], v[5], v[6], v[7]);
    dft4_si2<FWD>(v[8], v[9], v[10], v[11]);
    dft4<FWD>(v[12], v[13], v[14], v[15]);
    // v[4*k1 + k2] holds Y[k1 + 4*k2]: transpose the 4x4 index
    float2 y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = y[i];
}

template <int R, bool FWD>
__host__ __device__ __forceinline__ void dft(float2* v)
{
    if constexpr (R == 2) dft2<FWD>(v[0], v[1]);
    else if constexpr (R == 3) dft3<FWD>(v[0], v[1], v[2]);
    else if constexpr (R == 4) dft4<FWD>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 5) dft5<FWD>(v);
    else if constexpr (R == 8) dft8<FWD>(v);
    else if constexpr (R == 16) dft16<FWD>(v);
}

#ifdef __CUDACC__

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

// Padded shared-memory index of element i of a line: one gap every 16 values
// keeps the stride-R writes of early stages free of bank conflicts.
__host__ __device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

// ---------------------------------------------------------------------------
// TMA (bulk asynchronous copy) and mbarrier primitives, in inline PTX.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Self-check build (FB_FFT_SELFCHECK): every copy validates its addresses and
// size first; a violation is recorded in err[1..3] (kind, address, bytes),
// err[0] is set and the copy is skipped (its wait then times out cleanly).
#ifdef FB_FFT_SELFCHECK
__device__ __forceinline__ bool selfcheck_bad(int* err, int kind, const void* g, const void* s, unsigned bytes,
                                              unsigned galign, unsigned salign)
{
    const bool bad = ((unsigned long long)g % galign) != 0 || (s && (smem_u32(s) % salign) != 0) ||
                     (bytes % 16) != 0 || bytes == 0;
    if (bad && atomicCAS(err + 1, 0, kind) == 0) {
        err[2] = (int)((unsigned long long)g & 0x7fffffff);
        err[3] = (int)bytes;
        atomicExch(err, 2);
    }
    return bad;
}
#define FB_SELFCHECK(err, kind, g, s, bytes, ga, sa) \
    if (selfcheck_bad(err, kind, g, s, bytes, ga, sa)) return
#else
#define FB_SELFCHECK(err, kind, g, s, bytes, ga, sa) (void)0
#endif

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Programmatic dependent launch.  Every line-pass kernel lets the next pass
// on its stream start its CTAs (prologue: barriers, shared-memory set-up) as
// soon as SMs free up, and itself waits, before its first global access, until
// the previous pass has completed and its writes are visible.  Launched
// without the attribute, both are no-ops.
__device__ __forceinline__ void pdl_start()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Make this thread's generic-proxy shared-memory writes visible to the TMA engine.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity; give up after kWaitLimitNs.
constexpr unsigned long long kWaitLimitNs = 1000000000ULL;
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitLimitNs) return false;
    return true;
}
// L2 policy for data read once: its lines go first when L2 needs room.
__device__ __forceinline__ unsigned long long l2_evict_first_policy()
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// L2 policy for data the next pass of the same exec reads: its lines stay
// while others can go.
__device__ __forceinline__ unsigned long long l2_evict_last_policy()
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// global -> shared, contiguous bytes; completion counted on `bar`; with
// `hint`, the source lines take the L2 policy `pol`.
__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                             int* err = nullptr, bool hint = false, unsigned long long pol = 0)
{
    if (err) FB_SELFCHECK(err, 11, src, dst, bytes, 16, 16);
    if (hint)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
            "%4;" ::"r"(smem_u32(dst)),
            "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
            : "memory");
    else
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(dst)),
                     "l"(src), "r"(bytes), "r"(smem_u32(bar))
                     : "memory");
}
// shared -> global, contiguous bytes; tracked by the issuing thread's bulk
// group; with `hint`, the written lines take the L2 policy `pol`.
__device__ __forceinline__ void bulk_store_1d(void* dst, const void* src, unsigned bytes, int* err = nullptr,
                                              bool hint = false, unsigned long long pol = 0)
{
    if (err) FB_SELFCHECK(err, 12, dst, src, bytes, 16, 16);
    if (hint)
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
                     "r"(smem_u32(src)), "r"(bytes), "l"(pol)
                     : "memory");
    else
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                     "r"(bytes)
                     : "memory");
}
// 3-D tiled tensor copies (coordinates innermost first).
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z, unsigned long long* bar,
                                            int* err = nullptr, bool hint = false, unsigned long long pol = 0)
{
    if (err) FB_SELFCHECK(err, 13, tmap, dst, 16u, 64, 128);
    if (hint)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
            "{%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
            "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)), "l"(pol)
            : "memory");
    else
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];" ::"r"(smem_u32(dst)),
            "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
            : "memory");
}
__device__ __forceinline__ void tma_store_3d(const void* tmap, int x, int y, int z, const void* src,
                                             int* err = nullptr, bool hint = false, unsigned long long pol = 0)
{
    if (err) FB_SELFCHECK(err, 14, tmap, src, 16u, 64, 128);
    if (hint)
        asm volatile(
            "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group.L2::cache_hint [%0, {%1, %2, %3}], [%4], "
            "%5;" ::"l"(tmap),
            "r"(x), "r"(y), "r"(z), "r"(smem_u32(src)), "l"(pol)
            : "memory");
    else
        asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                         tmap),
                     "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                     : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

struct TileIdx {
    long long o, c0;
    int Tv;
};


__device__ __forceinline__ TileIdx tile_index(const PassDesc& d, long long tile)
{
    TileIdx ti;
    ti.o = tile / d.tiles_per_o;
    ti.c0 = (tile - ti.o * d.tiles_per_o) << d.logT;
    const long long rem = d.C - ti.c0;
    const int T = 1 << d.logT;
    ti.Tv = rem < T ? (int)rem : T;
    return ti;
}

// Global base of the input / output a tile reads or writes.  With an offset
// table (batched uneven lengths), transform x starts at off[x]: x is the line
// for contiguous layouts, the outer index o for strided ones.
__device__ __forceinline__ const float2* tile_in_base(const PassDesc& d, const TileIdx& ti, bool strided)
{
    if (d.off_in) return d.in + (strided ? d.off_in[ti.o] + ti.c0 : 0);
    return d.in + ti.o * d.in_so + ti.c0 * d.in_sc;
}
__device__ __forceinline__ float2* tile_out_base(const PassDesc& d, const TileIdx& ti, bool strided)
{
    if (d.off_out) return d.out + (strided ? d.off_out[ti.o] + ti.c0 : 0);
    return d.out + ti.o * d.out_so + ti.c0 * d.out_sc;
}
// Start of line t of a contiguous-layout tile.
__device__ __forceinline__ const float2* line_in(const PassDesc& d, const TileIdx& ti, const float2* base, int t)
{
    return d.off_in ? d.in + d.off_in[ti.c0 + t] : base + (long long)t * d.in_sc;
}
__device__ __forceinline__ float2* line_out(const PassDesc& d, const TileIdx& ti, float2* base, int t)
{
    return d.off_out ? d.out + d.off_out[ti.c0 + t] : base + (long long)t * d.out_sc;
}

// Thread 0: start the TMA loads of one tile into a landing buffer.
// n-fast tiles are contiguous (line stride == L) and land as [t][n];
// c-fast tiles land as [n][t] by 3-D boxes of T x box_rows (zero fill past C).
__device__ __forceinline__ void issue_tile_load(const PassDesc& d, const CUtensorMap* tm_in, long long tile,
                                                float2* land, unsigned long long* bar)
{
    const TileIdx ti = tile_index(d, tile);
    const int L = d.L, T = 1 << d.logT;
    if (!d.in_tfast) {
        const unsigned bytes = (unsigned)(ti.Tv * L) * 8u;
        mbar_arrive_expect_tx(bar, bytes + d.debug_extra_tx);
        bulk_load_1d(land, d.in + ti.o * d.in_so + ti.c0 * d.in_sc, bytes, bar, d.err);
    } else {
        mbar_arrive_expect_tx(bar, (unsigned)(T * L) * 8u + d.debug_extra_tx);
        for (int n0 = 0; n0 < L; n0 += d.box_rows)
            tma_load_3d(land + n0 * T, tm_in, (int)ti.c0, n0, (int)ti.o, bar, d.err);
    }
}
// Thread 0: start the TMA stores of one finished tile from its buffer.
__device__ __forceinline__ void issue_tile_store(const PassDesc& d, const CUtensorMap* tm_out, long long tile,
                                                 const float2* land)
{
    const TileIdx ti = tile_index(d, tile);
    const int L = d.L, T = 1 << d.logT;
    if (!d.out_tfast) {
        bulk_store_1d(d.out + ti.o * d.out_so + ti.c0 * d.out_sc, land, (unsigned)(ti.Tv * L) * 8u, d.err);
    } else {
        for (int k0 = 0; k0 < L; k0 += d.box_rows) tma_store_3d(tm_out, (int)ti.c0, k0, (int)ti.o, land + k0 * T, d.err);
    }
    bulk_commit();
}

// Per-thread asynchronous copies (cp.async, 8 bytes each): any gather
// pattern, completion tracked per thread by commit groups.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Tile copies by the whole CTA.  Contiguous tiles ([t][n]): THREADS >> logT
// threads per line (T <= THREADS, both powers of two), consecutive threads on
// consecutive elements of one line, so a thread finds its line once per tile
// (one offset-table read) and needs no division.  Strided tiles ([n][t]):
// consecutive threads on consecutive lines.
template <int THREADS, bool ASYNC>
__device__ __forceinline__ void tile_copy_in(const PassDesc& d, const TileIdx& ti, float2* land)
{
    const int L = d.L, logT = d.logT, T = 1 << logT;
    const float2* gin = tile_in_base(d, ti, d.in_tfast != 0);
    const long long sn = d.in_sn;
    int t, n, step;
    float2* dst;
    const float2* src;
    int dstep;
    if (!d.in_tfast) {
        const int lgt = ilog2(THREADS) - logT;  // log2 threads per line
        t = threadIdx.x >> lgt;
        n = threadIdx.x & ((1 << lgt) - 1);
        step = 1 << lgt;
        if (t >= ti.Tv) return;
        src = line_in(d, ti, gin, t) + n * sn;
        dst = land + t * L + n;
        dstep = step;
    } else {
        t = threadIdx.x & (T - 1);
        n = threadIdx.x >> logT;
        step = THREADS >> logT;
        if (t >= ti.Tv) return;
        src = gin + n * sn + t;
        dst = land + (n << logT) + t;
        dstep = step << logT;
    }
    const long long sstep = step * sn;
    for (; n < L; n += step, src += sstep, dst += dstep) {
        if constexpr (ASYNC)
            cp_async8(dst, src);
        else
            *dst = *src;
    }
}
// Plain-copy fallback (misaligned bases, odd strides).
template <int THREADS>
__device__ __forceinline__ void plain_tile_load(const PassDesc& d, const TileIdx& ti, float2* land)
{
    tile_copy_in<THREADS, false>(d, ti, land);
}
// The same copies issued as cp.async (the caller commits and waits).
template <int THREADS>
__device__ __forceinline__ void async_tile_load(const PassDesc& d, const TileIdx& ti, float2* land)
{
    tile_copy_in<THREADS, true>(d, ti, land);
}
template <int THREADS>
__device__ __forceinline__ void plain_tile_store(const PassDesc& d, const TileIdx& ti, const float2* land)
{
    const int L = d.L, logT = d.logT, T = 1 << logT;
    float2* gout = tile_out_base(d, ti, d.out_tfast != 0);
    const long long sk = d.out_sk;
    int t, k, step, sstep_l;
    const float2* src;
    float2* dst;
    if (!d.out_tfast) {
        const int lgt = ilog2(THREADS) - logT;
        t = threadIdx.x >> lgt;
        k = threadIdx.x & ((1 << lgt) - 1);
        step = 1 << lgt;
        if (t >= ti.Tv) return;
        dst = line_out(d, ti, gout, t) + k * sk;
        src = land + t * L + k;
        sstep_l = step;
    } else {
        t = threadIdx.x & (T - 1);
        k = threadIdx.x >> logT;
        step = THREADS >> logT;
        if (t >= ti.Tv) return;
        dst = gout + k * sk + t;
        src = land + (k << logT) + t;
        sstep_l = step << logT;
    }
    const long long dstep = step * sk;
    for (; k < L; k += step, src += sstep_l, dst += dstep) *dst = *src;
}

// One Stockham stage for the whole tile.  Threads cover butterflies (t, j):
// t-fast mapping puts consecutive threads on consecutive lines (conflict-free
// on the [n][t] landing layout), j-fast on consecutive j.  Stage 0 reads the
// landing buffer, the last stage writes the tile's output layout back into it
// (with the four-step twiddle and the 1/N scale applied), the stages between
// work in place on the padded work buffer.
enum StagePos { kPosOnly = 0, kPosFirst = 1, kPosMid = 2, kPosLast = 3 };
__host__ __device__ constexpr bool last_pos(int pos) { return pos == kPosOnly || pos == kPosLast; }

template <int R, int THREADS, bool FWD, int POS, int E = kElemsPerThread, bool PP = false>
__device__ __forceinline__ void stage(const PassDesc& d, int st, float2* land, float2* work, int Tv, int c0,
                                      float2* work2 = nullptr)
{
    // PP: two work buffers; stage st writes buffer st & 1 and reads the other,
    // so a middle stage needs no barrier between its reads and its writes.
    float2* wr = work;
    const float2* rd = work;
    if constexpr (PP) {
        wr = (st & 1) ? work2 : work;
        rd = (st & 1) ? work : work2;
    }
    // Every descriptor field is read here, before the stage stores anything:
    // the descriptor may sit in shared memory, and a later read would have to
    // be repeated after each store to the tile buffers.
    const int Ns = d.ns[st];
    const unsigned nsm = d.ns_mag[st];  // ceil(2^32 / Ns): j mod Ns without a division (Ns > 1)
    const float2* twb = d.tw + d.twoff[st];
    const int logT = d.logT, L = d.L, LS = d.LS;
    const bool in_tf = d.in_tfast != 0, out_tf = d.out_tfast != 0;
    const bool ptw = last_pos(POS) && d.ptw != 0;
    const int ptw_log = d.ptw_log;
    const float2* ptw_hi = d.ptw_hi;
    const float2* ptw_lo = d.ptw_lo;
    const float scale = (last_pos(POS) && d.apply_scale) ? d.scale : 1.0f;
    constexpr int Q = (E + R - 1) / R;
    constexpr bool first = POS == kPosOnly || POS == kPosFirst;
    constexpr bool last = POS == kPosOnly || POS == kPosLast;
    const bool tfast = (first && in_tf) || (last && out_tf);
    const int tid = threadIdx.x;
    const int T = 1 << logT;
    const int G = THREADS >> logT;  // threads per line
    const int LR = L / R;
    int t, jb;
    if (tfast) {
        t = tid & (T - 1);
        jb = tid >> logT;
    } else {
        t = tid >> (ilog2(THREADS) - logT);  // tid / G, G a power of two
        jb = tid & (G - 1);
    }
    const bool tok = t < Tv;
    float2 v[Q][R];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int j = jb + q * G;
        if (tok && j < LR) {
            if constexpr (first) {
                if (in_tf) {
#pragma unroll
                    for (int r = 0; r < R; ++r) v[q][r] = land[((j + r * LR) << logT) + t];
                } else {
#pragma unroll
                    for (int r = 0; r < R; ++r) v[q][r] = land[t * L + j + r * LR];
                }
            } else {
                const float2* p = rd + t * LS;
#pragma unroll
                for (int r = 0; r < R; ++r) v[q][r] = p[spad(j + r * LR)];
            }
        } else {
            // defined on every path: loaded and used under the same condition,
            // which the register allocator cannot prove, the values would
            // otherwise stay live around the tile loop
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = make_float2(0.f, 0.f);
        }
    }
    if constexpr (first == last && (!PP || first)) __syncthreads();  // reads and writes share one buffer
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int j = jb + q * G;
        if (tok && j < LR) {
            const int k = first ? 0 : j - (int)__umulhi((unsigned)j, nsm) * Ns;
            if (!first) {
                const float2* tw = twb + k;
#pragma unroll
                for (int r = 1; r < R; ++r) v[q][r] = twmul<FWD>(v[q][r], __ldg(tw + (r - 1) * Ns));
            }
            dft<R, FWD>(v[q]);
            const int base = (j - k) * R + k;
            if constexpr (!last) {
                float2* p = wr + t * LS;
#pragma unroll
                for (int r = 0; r < R; ++r) p[spad(base + r * Ns)] = v[q][r];
            } else {
                const unsigned c = (unsigned)(c0 + t);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int kk = base + r * Ns;
                    float2 y = v[q][r];
                    if (ptw) {
                        const unsigned m = c * (unsigned)kk;  // < N < 2^31
                        const float2 w = cmul(__ldg(ptw_hi + (m >> ptw_log)), __ldg(ptw_lo + (m & ((1u << ptw_log) - 1))));
                        y = twmul<FWD>(y, w);
                    }
                    y = scale * y;
                    if (out_tf)
                        land[(kk << logT) + t] = y;
                    else
                        land[t * L + kk] = y;
                }
            }
        }
    }
}

template <int THREADS, bool FWD, int POS, int E>
__device__ __forceinline__ void run_stage(const PassDesc& d, int st, float2* land, float2* work, int Tv, int c0)
{
    switch (d.radix[st]) {
    case 16: stage<16, THREADS, FWD, POS, E>(d, st, land, work, Tv, c0); break;
    case 8: stage<8, THREADS, FWD, POS, E>(d, st, land, work, Tv, c0); break;
    case 5: stage<5, THREADS, FWD, POS, E>(d, st, land, work, Tv, c0); break;
    case 4: stage<4, THREADS, FWD, POS, E>(d, st, land, work, Tv, c0); break;
    case 3: stage<3, THREADS, FWD, POS, E>(d, st, land, work, Tv, c0); break;
    default: stage<2, THREADS, FWD, POS, E>(d, st, land, work, Tv, c0); break;
    }
}

// Power-of-two schedules, fixed at compile time.  log2 L = 4a + b: a radix-16
// stages and, when b > 0, one radix-2^b stage.  Two-stage schedules run the
// radix-16 stage first (every shared-memory phase then touches G consecutive
// values per line, which the row padding keeps conflict free); longer ones run
// the small radix first, where stage 0's lack of twiddles offsets its extra
// butterflies per thread.
__host__ __device__ constexpr int pow2_nst(int lg) { return lg / 4 + (lg % 4 ? 1 : 0); }
__host__ __device__ constexpr bool pow2_rem_first(int lg) { return (lg % 4) != 0 && pow2_nst(lg) >= 3; }
__host__ __device__ constexpr int pow2_radix(int lg, int s)
{
    return (lg % 4) == 0 ? 16
                         : (pow2_rem_first(lg) ? (s == 0 ? (1 << (lg % 4)) : 16)
                                               : (s == pow2_nst(lg) - 1 ? (1 << (lg % 4)) : 16));
}
// Ns before stage s (the product of the earlier radices).
__host__ __device__ constexpr int pow2_ns(int lg, int s)
{
    return s == 0 ? 1 : pow2_radix(lg, s - 1) * pow2_ns(lg, s - 1);
}

// The generic line pass: any 5-smooth L <= 4096, stage radices read from the
// descriptor at run time.  Persistent CTAs walk tiles blockIdx.x, +gridDim.x,
// ...; with TMA on (d.async_io), tile i+1 streams into the second landing
// buffer while tile i is transformed, and finished tiles leave by TMA stores.
template <int THREADS, bool FWD>
__global__ void __launch_bounds__(THREADS, 1) k_fft_generic(const __grid_constant__ LineArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // 128-byte aligned base (the size includes 128 bytes of slack for this)
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);  // 2 mbarriers
    float2* land0 = reinterpret_cast<float2*>(smem_raw + 128);
    const bool async = a.d.async_io != 0;
    float2* work = land0 + (async ? 2 : 1) * a.d.land_stride;
    const long long step = gridDim.x;
    // The descriptor, copied to shared memory once: field reads and the
    // dynamically indexed stage tables then never touch local memory.
    __shared__ PassDesc sd;
    {
        const int* src = reinterpret_cast<const int*>(&a.d);
        int* dst = reinterpret_cast<int*>(&sd);
        for (int w = threadIdx.x; w < (int)(sizeof(PassDesc) / 4); w += THREADS) dst[w] = src[w];
    }
    __syncthreads();
    pdl_start();
    const PassDesc& d = sd;
    if (async && threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        if (blockIdx.x < d.ntiles) issue_tile_load(d, &a.tm_in, blockIdx.x, land0, &bar[0]);
        if (blockIdx.x + step < d.ntiles)
            issue_tile_load(d, &a.tm_in, blockIdx.x + step, land0 + d.land_stride, &bar[1]);
    }
    __syncthreads();
    int i = 0;
    for (long long tile = blockIdx.x; tile < d.ntiles; tile += step, ++i) {
        const TileIdx ti = tile_index(d, tile);
        const int buf = async ? (i & 1) : 0;
        float2* land = land0 + buf * d.land_stride;
        const int c0 = (int)ti.c0;
        if (async) {
            const bool bad = !mbar_wait_bounded(&bar[buf], (unsigned)(i >> 1) & 1u);
            if (__syncthreads_or(bad)) {
                if (threadIdx.x == 0) {
                    atomicExch(d.err, 1);
                    bulk_wait_all();
                    if (i == 0 && tile + step < d.ntiles) mbar_wait_bounded(&bar[1], 0);
                }
                return;
            }
        } else {
            plain_tile_load<THREADS>(d, ti, land);
            __syncthreads();
        }
        if (d.nst == 1)
            run_stage<THREADS, FWD, kPosOnly, kGenericElems>(d, 0, land, work, ti.Tv, c0);
        else
            run_stage<THREADS, FWD, kPosFirst, kGenericElems>(d, 0, land, work, ti.Tv, c0);
        if (async && d.nst == 1) fence_proxy_async();
        __syncthreads();
        // The previous tile's store has had a stage to drain: recycle its
        // buffer for the next tile's load.
        if (async && i >= 1 && threadIdx.x == 0 && tile + step < d.ntiles) {
            bulk_wait_read_all();
            issue_tile_load(d, &a.tm_in, tile + step, land0 + (buf ^ 1) * d.land_stride, &bar[buf ^ 1]);
        }
        for (int s = 1; s < d.nst; ++s) {
            if (s == d.nst - 1)
                run_stage<THREADS, FWD, kPosLast, kGenericElems>(d, s, land, work, ti.Tv, c0);
            else
                run_stage<THREADS, FWD, kPosMid, kGenericElems>(d, s, land, work, ti.Tv, c0);
            if (async && s == d.nst - 1) fence_proxy_async();
            __syncthreads();
        }
        if (async) {
            if (threadIdx.x == 0) issue_tile_store(d, &a.tm_out, tile, land);
        } else {
            plain_tile_store<THREADS>(d, ti, land);
            __syncthreads();
        }
    }
    if (async && threadIdx.x == 0) bulk_wait_all();
}

// Run-time dispatch over the odd radices only (5, 3).
template <int THREADS, bool FWD, int POS, int E, bool PP = false>
__device__ __forceinline__ void run_odd_stage(const PassDesc& d, int st, float2* land, float2* work, int Tv, int c0,
                                              float2* work2 = nullptr)
{
    if (d.radix[st] == 5)
        stage<5, THREADS, FWD, POS, E, PP>(d, st, land, work, Tv, c0, work2);
    else
        stage<3, THREADS, FWD, POS, E, PP>(d, st, land, work, Tv, c0, work2);
}
// Compile-time power-of-two prefix of a mixed schedule (stage S < pow2_nst(LG2)).
template <int THREADS, bool FWD, int LG2, int S, int E, bool PP = false>
__device__ __forceinline__ void mixed_p2_stages(const PassDesc& d, float2* land, float2* work, int Tv, int c0,
                                                float2* work2 = nullptr)
{
    if constexpr (S < pow2_nst(LG2)) {
        constexpr int R = pow2_radix(LG2, S);
        stage<R, THREADS, FWD, S == 0 ? kPosFirst : kPosMid, E, PP>(d, S, land, work, Tv, c0, work2);
        __syncthreads();
        mixed_p2_stages<THREADS, FWD, LG2, S + 1, E, PP>(d, land, work, Tv, c0, work2);
    }
}

// The mixed line pass: L = 2^LG2 * 3^b * 5^c with b + c >= 1.  Stages: the
// power-of-two radices (compile time), then the 5s, then the 3s (run time).
// Same tile walk and TMA pipeline as the generic kernel.
template <int THREADS, bool FWD, int LG2>
__global__ void __launch_bounds__(THREADS, 1) k_fft_mixed(const __grid_constant__ LineArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);
    float2* land0 = reinterpret_cast<float2*>(smem_raw + 128);
    const bool async = a.d.async_io != 0;
    float2* work = land0 + (async ? 2 : 1) * a.d.land_stride;
    const long long step = gridDim.x;
    __shared__ PassDesc sd;
    {
        const int* src = reinterpret_cast<const int*>(&a.d);
        int* dst = reinterpret_cast<int*>(&sd);
        for (int w = threadIdx.x; w < (int)(sizeof(PassDesc) / 4); w += THREADS) dst[w] = src[w];
    }
    __syncthreads();
    pdl_start();
    const PassDesc& d = sd;
    constexpr int E = kMixedElems;
    constexpr int NP2 = pow2_nst(LG2);
    if (async && threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        if (blockIdx.x < d.ntiles) issue_tile_load(d, &a.tm_in, blockIdx.x, land0, &bar[0]);
        if (blockIdx.x + step < d.ntiles)
            issue_tile_load(d, &a.tm_in, blockIdx.x + step, land0 + d.land_stride, &bar[1]);
    }
    __syncthreads();
    int i = 0;
    for (long long tile = blockIdx.x; tile < d.ntiles; tile += step, ++i) {
        const TileIdx ti = tile_index(d, tile);
        const int buf = async ? (i & 1) : 0;
        float2* land = land0 + buf * d.land_stride;
        const int c0 = (int)ti.c0;
        if (async) {
            const bool bad = !mbar_wait_bounded(&bar[buf], (unsigned)(i >> 1) & 1u);
            if (__syncthreads_or(bad)) {
                if (threadIdx.x == 0) {
                    atomicExch(d.err, 1);
                    bulk_wait_all();
                    if (i == 0 && tile + step < d.ntiles) mbar_wait_bounded(&bar[1], 0);
                }
                return;
            }
        } else {
            plain_tile_load<THREADS>(d, ti, land);
            __syncthreads();
        }
        int s0 = NP2;
        if constexpr (NP2 > 0) {
            mixed_p2_stages<THREADS, FWD, LG2, 0, E>(d, land, work, ti.Tv, c0);
        } else {
            if (d.nst == 1)
                run_odd_stage<THREADS, FWD, kPosOnly, E>(d, 0, land, work, ti.Tv, c0);
            else
                run_odd_stage<THREADS, FWD, kPosFirst, E>(d, 0, land, work, ti.Tv, c0);
            if (async && d.nst == 1) fence_proxy_async();
            __syncthreads();
            s0 = 1;
        }
        if (async && i >= 1 && threadIdx.x == 0 && tile + step < d.ntiles) {
            bulk_wait_read_all();
            issue_tile_load(d, &a.tm_in, tile + step, land0 + (buf ^ 1) * d.land_stride, &bar[buf ^ 1]);
        }
        for (int s = s0; s < d.nst; ++s) {
            if (s == d.nst - 1)
                run_odd_stage<THREADS, FWD, kPosLast, E>(d, s, land, work, ti.Tv, c0);
            else
                run_odd_stage<THREADS, FWD, kPosMid, E>(d, s, land, work, ti.Tv, c0);
            if (async && s == d.nst - 1) fence_proxy_async();
            __syncthreads();
        }
        if (async) {
            if (threadIdx.x == 0) issue_tile_store(d, &a.tm_out, tile, land);
        } else {
            plain_tile_store<THREADS>(d, ti, land);
            __syncthreads();
        }
    }
    if (async && threadIdx.x == 0) bulk_wait_all();
}

// (Power-of-two factors up to 16 run two CTAs per SM, which overlap one
// another's barriers: 2..16 fit 128 registers; odd lengths spill about 0.5 KB
// there and still measured 1.2x faster than at one CTA per SM.  Larger
// factors need more registers and run one CTA per SM.)
// The mixed line pass over several jobs (MultiArgs): persistent CTAs walk the
// global tiles blockIdx.x, +gridDim.x, ...; a tile's job is found by advancing
// through the prefix table (tiles only grow).  Two landing buffers, each with
// its tile's descriptor in shared memory: while tile i is transformed, every
// thread's cp.async copies bring tile i+1 through its job's offset table.
// Two work buffers: the stages alternate between them (one barrier per stage).
template <int THREADS, bool FWD, int LG2>
__global__ void __launch_bounds__(THREADS, (LG2 <= 4 ? 2 : 1)) k_fft_mixed_multi(const __grid_constant__ MultiArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    float2* land0 = reinterpret_cast<float2*>(smem_raw + 128);
    float2* work = land0 + 2 * a.land_max;
    float2* work2 = work + a.work_max;  // second work buffer: middle stages alternate
    __shared__ PassDesc sd[2];  // sd[b]: descriptor of the tile in landing buffer b
    constexpr int E = kMixedElems;
    constexpr int NP2 = pow2_nst(LG2);
    const long long total = a.tile_start[a.njobs];
    const long long step = gridDim.x;
    auto copy_desc = [&](int job, int b) {
        const int* src = reinterpret_cast<const int*>(&a.d[job]);
        int* dst = reinterpret_cast<int*>(&sd[b]);
        for (int w = threadIdx.x; w < (int)(sizeof(PassDesc) / 4); w += THREADS) dst[w] = src[w];
    };
    pdl_start();
    int j = 0;
    long long g = blockIdx.x;
    if (g < total) {
        while (j + 1 < a.njobs && g >= a.tile_start[j + 1]) ++j;
        copy_desc(j, 0);
        __syncthreads();
        async_tile_load<THREADS>(sd[0], tile_index(sd[0], g - a.tile_start[j]), land0);
        cp_async_commit();
    }
    long long jstart = a.tile_start[j];
    for (int i = 0; g < total; g += step, ++i) {
        const int b = i & 1;
        const long long gl = g - jstart;  // this tile within its job
        const long long gn = g + step;
        if (gn < total) {  // the next tile's job and descriptor, then its copies
            while (j + 1 < a.njobs && gn >= a.tile_start[j + 1]) ++j;
            jstart = a.tile_start[j];
            copy_desc(j, b ^ 1);
            __syncthreads();
            async_tile_load<THREADS>(sd[b ^ 1], tile_index(sd[b ^ 1], gn - jstart), land0 + (b ^ 1) * a.land_max);
            cp_async_commit();
            cp_async_wait<1>();  // this tile's copies have landed (the next tile's may still fly)
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const PassDesc& d = sd[b];
        float2* land = land0 + b * a.land_max;
        const TileIdx ti = tile_index(d, gl);
        const int c0 = (int)ti.c0;
        int s0 = NP2;
        if constexpr (NP2 > 0) {
            mixed_p2_stages<THREADS, FWD, LG2, 0, E, true>(d, land, work, ti.Tv, c0, work2);
        } else {
            if (d.nst == 1)
                run_odd_stage<THREADS, FWD, kPosOnly, E, true>(d, 0, land, work, ti.Tv, c0, work2);
            else
                run_odd_stage<THREADS, FWD, kPosFirst, E, true>(d, 0, land, work, ti.Tv, c0, work2);
            __syncthreads();
            s0 = 1;
        }
        for (int s = s0; s < d.nst; ++s) {
            if (s == d.nst - 1)
                run_odd_stage<THREADS, FWD, kPosLast, E, true>(d, s, land, work, ti.Tv, c0, work2);
            else
                run_odd_stage<THREADS, FWD, kPosMid, E, true>(d, s, land, work, ti.Tv, c0, work2);
            __syncthreads();
        }
        plain_tile_store<THREADS>(d, ti, land);
        __syncthreads();  // buffer b and sd[b] are free for the tile after next
    }
}

// A kernel's table entry: its pointer, CTA size and a printable name.
template <int THREADS>
LineKernel make_entry(void (*fn)(LineArgs), bool fwd, int lg, int io)
{
    LineKernel k;
    k.fn = fn;
    k.threads = THREADS;
    k.fwd = fwd;
    k.lg = lg;
    k.io = io;
    return k;
}

template <int THREADS, bool FWD>
LineKernel generic_entry()
{
    LineKernel k = make_entry<THREADS>(k_fft_generic<THREADS, FWD>, FWD, 0, -1);
    k.kind = 1;
    return k;
}
template <bool FWD, int LG2>
LineKernel mixed_entry()
{
    LineKernel k = make_entry<kMixedThreads>(k_fft_mixed<kMixedThreads, FWD, LG2>, FWD, LG2, -1);
    k.kind = 2;
    return k;
}

#endif  // __CUDACC__

}  // namespace fbfft
