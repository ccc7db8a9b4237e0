// fft_uneven.cuh -- the line pass of batched uneven lengths (fb_fft_plan_many):
// single-pass lines, four-step columns and four-step rows of any 5-smooth
// length up to 2048, power-of-two or not.  k_fft_uneven runs every pass of
// one phase of such a batch in one launch (phase 0: single passes and
// columns; phase 1: rows); k_fft_uneven_one (below) runs both phases in ONE
// launch, each row chunk after its columns.
//
// Jobs (one PassDesc per length group or four-step chunk, each with its own
// offset tables, strides, radix schedule and twiddle tables) sit in a device
// table; a device prefix table gives each job's first global tile.
// k_fft_uneven's persistent CTAs walk the global tiles blockIdx.x,
// +gridDim.x, ... (k_fft_uneven_one's claim them from a counter): the job of a
// tile is found by walking the prefix table forward (tiles only grow).
// Two landing buffers, each with its tile's descriptor in shared memory:
// while tile i is transformed, every thread's cp.async copies bring tile i+1
// (16-byte copies where the layout allows, else 8-byte).  The stages alternate
// between the work buffer and the tile's own landing buffer, so every stage
// needs one barrier; the last stage stores to global memory directly.  Stage
// radices come from the descriptor (8, 4, 2, 5, 3: at most 10 values of one
// thread in flight), which keeps the kernel at 64 registers and three
// buffers, four CTAs per SM.
#pragma once

#include "fft_device.cuh"

namespace fbfft {

constexpr int kUnevenThreads = 256;
constexpr int kUnevenElems = 8;                                 // values per thread and stage
constexpr int kUnevenCap = kUnevenThreads * kUnevenElems;       // values per tile (2048)
constexpr int kUnevenMaxLen = kUnevenCap;                       // longest line of a job

// Kernel argument: the job table and the tile prefix table (device memory,
// written once when the plan is built, or per launch by the request server)
// and the buffers of this exec.  A job's `in` / `out` fields hold element
// offsets into the buffer its in_buf / out_buf names, or (kind 3) addresses.
struct UnevenArgs {
    const PassDesc* jobs;   // [njobs]
    const int* tile_start;  // [njobs + 1]: first global tile of each job; [njobs] = all tiles
    const float2* in;       // buffer 0: the caller's input
    float2* out;            // buffer 1: the caller's output
    float2* scratch;        // buffer 2: the plan's four-step intermediate
    int njobs;
    int land_max;           // elements of one landing buffer (multiple of 16; holds a padded work tile too)
    int work_max;           // elements of the work buffer (multiple of 16)
    int scale_on;           // 1: jobs marked apply_scale multiply by their `scale`
    // One-launch form (k_fft_uneven_one) only: device counters, nsync of
    // them, zero between execs -- [0] tiles claimed, [1] CTAs finished,
    // [1 + s] finished tiles of dependency slot s (PassDesc::dep_post / dep).
    unsigned long long* sync;
    int nsync;
    int dep_extra;          // test hook: added to every dependency target (the waits then run out)
};

// Kernel argument of the inline form: the tables themselves (a.jobs and
// a.tile_start unused).  About 5.8 KB, well under the 32 KB parameter limit.
constexpr int kUnevenInlineJobs = 16;
struct UnevenInlineArgs {
    UnevenArgs a;
    PassDesc jobs[kUnevenInlineJobs];
    int tile_start[kUnevenInlineJobs + 1];
};

#ifdef __CUDACC__

// Tile t of job d: outer index o, first line c0, valid lines Tv (32-bit: a
// job has fewer than 2^31 tiles and lines).
struct UTileIdx {
    int o, c0, Tv;
};
__device__ __forceinline__ UTileIdx utile_index(const PassDesc& d, int tile)
{
    UTileIdx ti;
    const int tpo = (int)d.tiles_per_o;
    ti.o = (int)((unsigned)tile / (unsigned)tpo);
    ti.c0 = (tile - ti.o * tpo) << d.logT;
    const int rem = (int)d.C - ti.c0;
    const int T = 1 << d.logT;
    ti.Tv = rem < T ? rem : T;
    return ti;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

// A job's input / output base in this exec's buffers; kind 3: the field is
// the address itself (jobs of different requests in one server launch).
__device__ __forceinline__ const float2* ubuf_in(const UnevenArgs& a, const PassDesc& d)
{
    if (d.in_buf == 3) return d.in;
    const float2* b = d.in_buf == 0 ? a.in : (d.in_buf == 1 ? a.out : a.scratch);
    return b + (long long)reinterpret_cast<uintptr_t>(d.in);
}
__device__ __forceinline__ float2* ubuf_out(const UnevenArgs& a, const PassDesc& d)
{
    if (d.out_buf == 3) return d.out;
    float2* b = d.out_buf == 1 ? a.out : a.scratch;
    return b + (long long)reinterpret_cast<uintptr_t>(d.out);
}
// Global start of line (o, c) of the input / output (offset tables or strides).
__device__ __forceinline__ const float2* uline_in(const UnevenArgs& a, const PassDesc& d, int o, int c)
{
    const float2* in = ubuf_in(a, d);
    if (d.off_in) return in + (d.in_tfast ? d.off_in[o] + c : d.off_in[c]);
    return in + (long long)o * d.in_so + (long long)c * d.in_sc;
}
__device__ __forceinline__ float2* uline_out(const UnevenArgs& a, const PassDesc& d, int o, int c)
{
    float2* out = ubuf_out(a, d);
    if (d.off_out) return out + (d.out_tfast ? d.off_out[o] + c : d.off_out[c]);
    return out + (long long)o * d.out_so + (long long)c * d.out_sc;
}

// Copy tile ti of job d into `land` with cp.async (the caller commits and
// waits).  Contiguous lines land as [t][n]: 2^lgt threads per line (T <= 256
// lines, both powers of two), consecutive threads on consecutive values, so a
// thread finds its line once per tile.  Strided tiles land as [n][t]:
// consecutive threads on consecutive lines.  Pairs of values move as one
// 16-byte copy when every address of the tile is 16-byte aligned.
__device__ __forceinline__ void utile_load(const UnevenArgs& a, const PassDesc& d, const UTileIdx& ti, float2* land)
{
    constexpr int LGTH = 8;  // log2(kUnevenThreads)
    const int L = d.L, logT = d.logT, tid = threadIdx.x;
    if (!d.in_tfast) {
        const int lgt = LGTH - logT, t = tid >> lgt, step = 1 << lgt;
        if (t >= ti.Tv) return;
        const float2* src = uline_in(a, d, ti.o, ti.c0 + t);
        const int lrow = d.land_row ? d.land_row : L;
        float2* dst = land + t * lrow;
        if ((L & 1) == 0 && (lrow & 1) == 0 && ((uintptr_t)src & 15) == 0) {
            for (int n = 2 * (tid & (step - 1)); n < L; n += 2 * step) cp_async16(dst + n, src + n);
        } else {
            for (int n = tid & (step - 1); n < L; n += step) cp_async8(dst + n, src + n);
        }
    } else {
        const float2* base = uline_in(a, d, ti.o, ti.c0);
        const long long sn = d.in_sn;
        const int T = 1 << logT;
        if (logT >= 1 && (ti.Tv & 1) == 0 && (sn & 1) == 0 && ((uintptr_t)base & 15) == 0) {
            const int lg = logT - 1, t = 2 * (tid & ((1 << lg) - 1)), step = kUnevenThreads >> lg;
            if (t >= ti.Tv) return;
            for (int n = tid >> lg; n < L; n += step) cp_async16(land + n * T + t, base + n * sn + t);
        } else {
            const int t = tid & (T - 1), step = kUnevenThreads >> logT;
            if (t >= ti.Tv) return;
            for (int n = tid >> logT; n < L; n += step) cp_async8(land + n * T + t, base + n * sn + t);
        }
    }
}

// exp(-2 pi i m / N) from the job's two split four-step tables (m < N < 2^31).
__device__ __forceinline__ float2 uptw(const PassDesc& d, unsigned m)
{
    return cmul(__ldg(d.ptw_hi + (m >> d.ptw_log)), __ldg(d.ptw_lo + (m & ((1u << d.ptw_log) - 1))));
}

// A shared-memory value read with a volatile load (see ustage).
template <class T>
__device__ __forceinline__ T uvol(const T& x)
{
    return *const_cast<const volatile T*>(&x);
}

// One Stockham stage of radix R over the tile (see fft_device.cuh for the
// formula).  Buffers: stage 0 reads the landing buffer (the input layout) and
// writes the padded work buffer; from then on the tile's own landing buffer
// is free and serves as the second work buffer: stage st >= 1 reads the work
// buffer and writes the landing buffer when st is odd, the other way round
// when st is even, so no stage waits between its reads and its writes.  The
// last stage stores straight to global memory (coalesced in both output
// layouts), with the four-step twiddle and the scale applied.
template <int R, bool FWD, int POS>
__device__ __forceinline__ void ustage(const UnevenArgs& a, const PassDesc& d, int st, float2* land, float2* work,
                                       const UTileIdx& ti)
{
    constexpr int LGTH = 8;
    constexpr int Q = (kUnevenElems + R - 1) / R;
    constexpr bool first = POS == kPosFirst;
    constexpr bool last = POS == kPosLast;
    static_assert(POS == kPosFirst || POS == kPosMid || POS == kPosLast, "stage positions of the uneven kernel");
    const float2* rd = (st & 1) ? work : land;
    float2* wr = (st & 1) ? land : work;
    // Descriptor fields are read afresh in every stage (volatile loads), so
    // nothing derived from them stays live from one stage to the next.
    const int L = uvol(d.L), LS = uvol(d.LS), logT = uvol(d.logT);
    const int LR = L / R;
    const bool in_tf = first && uvol(d.in_tfast) != 0;
    const bool out_tf = last && uvol(d.out_tfast) != 0;
    // contiguous input with padded landing rows: the first stage too maps
    // threads across lines (its radix-R groups would otherwise fill a
    // half-warp at stride R)
    const int lrow = first ? uvol(d.land_row) : 0;
    const bool tfast = in_tf || out_tf || lrow != 0;
    const int tid = threadIdx.x;
    const int lgG = LGTH - logT, G = 1 << lgG;
    const int t = tfast ? (tid & ((1 << logT) - 1)) : (tid >> lgG);
    const int jb = tfast ? (tid >> logT) : (tid & (G - 1));
    const bool tok = t < ti.Tv;
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
                    const float2* p = land + t * (lrow ? lrow : L) + j;
#pragma unroll
                    for (int r = 0; r < R; ++r) v[q][r] = p[r * LR];
                }
            } else {
                const float2* p = rd + t * LS + j;
#pragma unroll
                for (int r = 0; r < R; ++r) v[q][r] = p[r * LR];
            }
        } else {
            // defined on every path: otherwise the register allocator sees the
            // values live around the tile loop (loaded and used under the same
            // condition, which it cannot prove) and keeps every radix's set
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = make_float2(0.f, 0.f);
        }
    }
    const int Ns = first ? 1 : uvol(d.ns[st]);
    const unsigned nsm = first ? 0u : (unsigned)uvol(d.ns_mag[st]);
    const float2* twb = d.tw + (first ? 0 : uvol(d.twoff[st]));
    float2* dst = nullptr;
    long long sk = 0;
    bool sc = false;
    if constexpr (last) {
        // line c0 + t of the output (contiguous output), or the tile's first
        // column plus t (strided output)
        dst = out_tf ? uline_out(a, d, ti.o, ti.c0) + t : uline_out(a, d, ti.o, ti.c0 + (tok ? t : 0));
        sk = out_tf ? d.out_sk : 1;
        sc = a.scale_on && d.apply_scale;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int j = jb + q * G;
        if (tok && j < LR) {
            const int k = first ? 0 : j - (int)__umulhi((unsigned)j, nsm) * Ns;
            if constexpr (!first) {
                // the factors are the powers w^r of w = w_{Ns R}^k (table entry
                // (r-1) Ns + k): radix 8 loads w and w^4 and forms the other five
                // by complex multiplies (at most three deep), radix 4 and 5 load w
                // and w^2 -- fewer loads from tables that mostly miss L1
                const float2* tw = twb + k;
                if constexpr (R == 8) {
                    const float2 w1 = __ldg(tw), w4 = __ldg(tw + 3 * Ns);
                    const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
                    v[q][1] = twmul<FWD>(v[q][1], w1);
                    v[q][2] = twmul<FWD>(v[q][2], w2);
                    v[q][3] = twmul<FWD>(v[q][3], w3);
                    v[q][4] = twmul<FWD>(v[q][4], w4);
                    v[q][5] = twmul<FWD>(v[q][5], cmul(w4, w1));
                    v[q][6] = twmul<FWD>(v[q][6], cmul(w4, w2));
                    v[q][7] = twmul<FWD>(v[q][7], cmul(w4, w3));
                } else if constexpr (R == 4 || R == 5) {
                    const float2 w1 = __ldg(tw), w2 = __ldg(tw + Ns);
                    v[q][1] = twmul<FWD>(v[q][1], w1);
                    v[q][2] = twmul<FWD>(v[q][2], w2);
                    v[q][3] = twmul<FWD>(v[q][3], cmul(w2, w1));
                    if constexpr (R == 5) v[q][4] = twmul<FWD>(v[q][4], cmul(w2, w2));
                } else {
#pragma unroll
                    for (int r = 1; r < R; ++r) v[q][r] = twmul<FWD>(v[q][r], __ldg(tw + (r - 1) * Ns));
                }
            }
            dft<R, FWD>(v[q]);
            const int base = (j - k) * R + k;
            if constexpr (!last) {
                float2* p = wr + t * LS + base;
#pragma unroll
                for (int r = 0; r < R; ++r) p[r * Ns] = v[q][r];
            } else {
                // last stage: Ns = L / R, so base = j and kk = j + r Ns.  The
                // four-step twiddle exp(-2 pi i c kk / N) is read from the split
                // tables for r = 0 and stepped by exp(-2 pi i c Ns / N) for the
                // rest (at most 7 products in a row): one gather per butterfly
                const unsigned c = (unsigned)(ti.c0 + t);
                const bool ptw = d.ptw != 0;
                float2 w = make_float2(1.f, 0.f), wstep = make_float2(1.f, 0.f);
                if (ptw && R > 1) wstep = uptw(d, c * (unsigned)Ns);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int kk = base + r * Ns;
                    float2 y = v[q][r];
                    if (ptw) {
                        w = r == 0 ? uptw(d, c * (unsigned)kk) : cmul(w, wstep);
                        y = twmul<FWD>(y, w);
                    }
                    if (sc) y = d.scale * y;
                    dst[kk * sk] = y;
                }
            }
        }
    }
}

// First or last stage: any radix of the schedule.
template <bool FWD, int POS>
__device__ __forceinline__ void ustage_any(const UnevenArgs& a, const PassDesc& d, int st, float2* land,
                                           float2* work, const UTileIdx& ti)
{
    switch (d.radix[st]) {
    case 8: ustage<8, FWD, POS>(a, d, st, land, work, ti); break;
    case 4: ustage<4, FWD, POS>(a, d, st, land, work, ti); break;
    case 5: ustage<5, FWD, POS>(a, d, st, land, work, ti); break;
    case 3: ustage<3, FWD, POS>(a, d, st, land, work, ti); break;
    case 2: ustage<2, FWD, POS>(a, d, st, land, work, ti); break;
    default:  // radix 1: a copy (length 1, and the stage that ends a one-radix schedule)
        ustage<1, FWD, POS>(a, d, st, land, work, ti);
        break;
    }
}
// Middle stages of radix R, from stage s while the schedule has that radix
// (schedules list their radices in the order 8, 4, 2, 5, 3).
template <int R, bool FWD>
__device__ __forceinline__ void ustage_run(const UnevenArgs& a, const PassDesc& d, int& s, int nst, float2* land,
                                           float2* work, const UTileIdx& ti)
{
    while (s < nst - 1 && d.radix[s] == R) {
        ustage<R, FWD, kPosMid>(a, d, s, land, work, ti);
        __syncthreads();
        ++s;
    }
}

// A word of the job or tile-prefix table: read-only global memory, or (INL)
// the kernel's own parameter, which takes plain generic loads.
template <bool INL>
__device__ __forceinline__ int utab(const int* p)
{
    if constexpr (INL)
        return *p;
    else
        return __ldg(p);
}

template <bool FWD, bool INL>
__device__ __forceinline__ void uneven_body(const UnevenArgs& a, const PassDesc* jobs, const int* tile_start)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    float2* land0 = reinterpret_cast<float2*>(smem_raw);
    float2* work = land0 + 2 * a.land_max;
    __shared__ PassDesc sd[2];  // sd[b]: descriptor of the tile in landing buffer b
    constexpr int TH = kUnevenThreads;
    const int total = utab<INL>(tile_start + a.njobs);
    const int step = gridDim.x;
    auto copy_desc = [&](int job, int b) {
        const int* src = reinterpret_cast<const int*>(jobs + job);
        int* dst = reinterpret_cast<int*>(&sd[b]);
        for (int w = threadIdx.x; w < (int)(sizeof(PassDesc) / 4); w += TH) dst[w] = utab<INL>(src + w);
    };
    pdl_start();
    int g = blockIdx.x;
    if (g >= total) return;
    int j = 0;
    while (g >= utab<INL>(tile_start + j + 1)) ++j;
    int jstart = utab<INL>(tile_start + j);
    copy_desc(j, 0);
    __syncthreads();
    utile_load(a, sd[0], utile_index(sd[0], g - jstart), land0);
    cp_async_commit();
    for (int i = 0; g < total; g += step, ++i) {
        const int b = i & 1;
        const int gl = g - jstart;  // this tile within its job
        const int gn = g + step;
        if (gn < total) {  // the next tile's job and descriptor, then its copies
            while (gn >= utab<INL>(tile_start + j + 1)) ++j;
            jstart = utab<INL>(tile_start + j);
            copy_desc(j, b ^ 1);
            __syncthreads();
            utile_load(a, sd[b ^ 1], utile_index(sd[b ^ 1], gn - jstart), land0 + (b ^ 1) * a.land_max);
            cp_async_commit();
            cp_async_wait<1>();  // this tile's copies have landed (the next tile's may still fly)
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const PassDesc& d = sd[b];
        float2* land = land0 + b * a.land_max;
        const UTileIdx ti = utile_index(d, gl);
        const int nst = d.nst;  // >= 2: the planner ends a one-radix schedule with a radix-1 copy
        ustage_any<FWD, kPosFirst>(a, d, 0, land, work, ti);
        __syncthreads();
        int s = 1;
        ustage_run<8, FWD>(a, d, s, nst, land, work, ti);
        ustage_run<4, FWD>(a, d, s, nst, land, work, ti);
        ustage_run<2, FWD>(a, d, s, nst, land, work, ti);
        ustage_run<5, FWD>(a, d, s, nst, land, work, ti);
        ustage_run<3, FWD>(a, d, s, nst, land, work, ti);
        ustage_any<FWD, kPosLast>(a, d, nst - 1, land, work, ti);
        __syncthreads();  // buffer b and sd[b] are free for the tile after next
    }
}

template <bool FWD>
__global__ void __launch_bounds__(kUnevenThreads, 4) k_fft_uneven(const __grid_constant__ UnevenArgs a)
{
    uneven_body<FWD, false>(a, a.jobs, a.tile_start);
}

// ---------------------------------------------------------------------------
// Every pass of a batched uneven exec in ONE launch.  The job table holds the
// single passes and four-step columns, then the four-step rows; a row reads
// what the columns of its chunk wrote, so it may start only once they are
// done.  Tiles are claimed in table order from a device counter (one atomic
// per tile, issued a tile ahead), not assigned round robin: a claimed tile
// always belongs to a running CTA, so a row tile waits only for column tiles
// already held by running CTAs, and a column tile never waits (a CTA claims
// in increasing order, so whatever it holds before a column tile is a column
// tile too).  No CTA can therefore wait on one that is not resident,
// whatever else shares the GPU.  A column tile, once stored, raises its
// chunk's counter (every thread fences its own stores, a barrier, then one
// release add, at the barrier after the CTA's next first stage); a row tile's
// inputs load once an acquire read sees the counter at the chunk's
// column-tile count.  Where the next tile's inputs are not ready when it is
// claimed, its copies wait until the current tile is done (bounded: past the
// limit the error word is set and the tile runs anyway).  The last CTA to
// finish zeroes the counters for the next exec.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Thread 0: whether the inputs of job `job` are ready.  `seen` is the last
// dependency slot this CTA found complete: counters only grow during an
// exec, and the acquire that found it complete (then a barrier) already
// orders every later load of the CTA, so that slot needs no further read.
__device__ __forceinline__ bool udeps_ready(const UnevenArgs& a, const PassDesc* job, int& seen)
{
    const int dep = __ldg(&job->dep);
    if (dep == 0 || dep == seen) return true;
    if (ld_acquire_u64(a.sync + 1 + dep) <
        (unsigned long long)__ldg(&job->dep_need) + (unsigned long long)a.dep_extra)
        return false;
    seen = dep;
    return true;
}
// Thread 0: wait until they are, at most kWaitLimitNs; past it set the error
// word.  Once the word is set (by any CTA) no wait lasts longer, so a launch
// whose waits cannot end still ends within about one limit.
__device__ __forceinline__ void udeps_wait(const UnevenArgs& a, const PassDesc* job, int* err, int& seen)
{
    if (udeps_ready(a, job, seen)) return;
    const unsigned long long t0 = global_ns();
    while (!udeps_ready(a, job, seen)) {
        if (*reinterpret_cast<volatile int*>(err) != 0) return;
        if (global_ns() - t0 > kWaitLimitNs) {
            atomicExch(err, 1);
            return;
        }
        __nanosleep(200);
    }
}

template <bool FWD>
__device__ __forceinline__ void uneven_body_one(const UnevenArgs& a)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    float2* land0 = reinterpret_cast<float2*>(smem_raw);
    float2* work = land0 + 2 * a.land_max;
    __shared__ PassDesc sd[2];  // sd[b]: descriptor of the tile in landing buffer b
    __shared__ int s_tk[2];     // claimed tickets, handed from thread 0 to the CTA
    __shared__ int s_ok;        // 1: the next tile's inputs are ready
    __shared__ int s_ok0;       // the same for the first tile (s_ok may change before every warp read it)
    __shared__ int s_last;      // 1: this CTA finished last
    constexpr int TH = kUnevenThreads;
    const int tid = threadIdx.x;
    const PassDesc* jobs = a.jobs;
    const int* tile_start = a.tile_start;
    const int total = __ldg(tile_start + a.njobs);
    auto copy_desc = [&](int job, int b) {
        const int* src = reinterpret_cast<const int*>(jobs + job);
        int* dst = reinterpret_cast<int*>(&sd[b]);
        for (int w = tid; w < (int)(sizeof(PassDesc) / 4); w += TH) dst[w] = __ldg(src + w);
    };
    pdl_start();
    if (tid == 0) {
        s_tk[0] = (int)atomicAdd(a.sync, 1ull);
        s_tk[1] = (int)atomicAdd(a.sync, 1ull);
    }
    __syncthreads();
    int g = s_tk[0], gn = s_tk[1];
    int jg = 0;              // job of tile g
    bool cur_loaded = false; // tile g's copies issued
    // A column tile is counted one tile late, at the barrier after the next
    // tile's first stage: a fence orders only the fencing thread's own
    // stores, so every thread fences its share of the counted tile's stores,
    // then the barrier, then one release add -- by then those stores have
    // drained and the fences cost little (fencing right after the stores
    // stalled every column tile).  Pending counts go out before any
    // dependency wait and after the last tile.
    int pend = 0;  // dependency slot + 1 of a finished column tile not yet counted
    int seen = 0;  // thread 0: the last dependency slot + 1 found complete
    auto flush = [&]() {
        if (pend) {
            __threadfence();
            __syncthreads();
            if (tid == 0) red_release_add_u64(a.sync + 1 + pend, 1ull);
            pend = 0;
        }
    };
    if (g < total) {
        while (g >= __ldg(tile_start + jg + 1)) ++jg;
        copy_desc(jg, 0);
        if (tid == 0) s_ok0 = udeps_ready(a, jobs + jg, seen) ? 1 : 0;
        __syncthreads();
        cur_loaded = s_ok0 != 0;
        if (cur_loaded) utile_load(a, sd[0], utile_index(sd[0], g - __ldg(tile_start + jg)), land0);
        cp_async_commit();
    }
    for (int i = 0; g < total; ++i) {
        const int b = i & 1;
        float2* land = land0 + b * a.land_max;
        const int gl = g - __ldg(tile_start + jg);  // this tile within its job
        if (!cur_loaded) {  // inputs not ready when it was claimed: wait, then copy
            flush();
            if (tid == 0) udeps_wait(a, jobs + jg, sd[b].err, seen);
            __syncthreads();
            utile_load(a, sd[b], utile_index(sd[b], gl), land);
            cp_async_commit();
        }
        // the ticket of the tile after next, used one iteration later
        unsigned long long claim = 0;
        if (tid == 0) claim = atomicAdd(a.sync, 1ull);
        bool next_loaded = false;
        int jn = jg;
        if (gn < total) {  // the next tile's job and descriptor, then its copies when its inputs are ready
            while (gn >= __ldg(tile_start + jn + 1)) ++jn;
            copy_desc(jn, b ^ 1);
            if (tid == 0) s_ok = udeps_ready(a, jobs + jn, seen) ? 1 : 0;
            __syncthreads();
            next_loaded = s_ok != 0;
            if (next_loaded)
                utile_load(a, sd[b ^ 1], utile_index(sd[b ^ 1], gn - __ldg(tile_start + jn)),
                           land0 + (b ^ 1) * a.land_max);
            cp_async_commit();
            cp_async_wait<1>();  // this tile's copies have landed (the next tile's may still fly)
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const PassDesc& d = sd[b];
        const UTileIdx ti = utile_index(d, gl);
        const int nst = d.nst;
        const int post = d.dep_post;
        ustage_any<FWD, kPosFirst>(a, d, 0, land, work, ti);
        if (pend) __threadfence();  // the previous column tile's stores (see flush)
        __syncthreads();
        if (tid == 0 && pend) red_release_add_u64(a.sync + 1 + pend, 1ull);
        pend = 0;
        int s = 1;
        ustage_run<8, FWD>(a, d, s, nst, land, work, ti);
        ustage_run<4, FWD>(a, d, s, nst, land, work, ti);
        ustage_run<2, FWD>(a, d, s, nst, land, work, ti);
        ustage_run<5, FWD>(a, d, s, nst, land, work, ti);
        ustage_run<3, FWD>(a, d, s, nst, land, work, ti);
        ustage_any<FWD, kPosLast>(a, d, nst - 1, land, work, ti);
        if (tid == 0) s_tk[i & 1] = (int)claim;
        __syncthreads();  // buffer b and sd[b] are free
        pend = post;
        g = gn;
        jg = jn;
        gn = s_tk[i & 1];
        cur_loaded = next_loaded;
    }
    flush();
    // the last CTA out zeroes the counters (every other CTA's atomics are
    // ordered before its finish count by the fences)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(a.sync + 1, 1ull) == (unsigned long long)gridDim.x - 1 ? 1 : 0;
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last)
        for (int k = tid; k < a.nsync; k += TH) a.sync[k] = 0ull;
}

template <bool FWD>
__global__ void __launch_bounds__(kUnevenThreads, 4) k_fft_uneven_one(const __grid_constant__ UnevenArgs a)
{
    uneven_body_one<FWD>(a);
}

// The same pass with its job and tile-prefix tables inside the kernel
// parameter (at most kUnevenInlineJobs jobs): a small batch then needs no
// copy of its tables to the device before it can start.
template <bool FWD>
__global__ void __launch_bounds__(kUnevenThreads, 4) k_fft_uneven_inline(const __grid_constant__ UnevenInlineArgs p)
{
    uneven_body<FWD, true>(p.a, p.jobs, p.tile_start);
}

#endif  // __CUDACC__

// Host side (fft_kernels_uneven.cu).
cudaError_t uneven_launch(bool forward, const UnevenArgs& a, long long grid, size_t smem, cudaStream_t stream);
cudaError_t uneven_occupancy(bool forward, size_t smem, int* blocks_per_sm);
cudaError_t uneven_launch_inline(bool forward, const UnevenInlineArgs& a, long long grid, size_t smem,
                                 cudaStream_t stream);
cudaError_t uneven_occupancy_inline(bool forward, size_t smem, int* blocks_per_sm);
cudaError_t uneven_launch_one(bool forward, const UnevenArgs& a, long long grid, size_t smem, cudaStream_t stream);
cudaError_t uneven_occupancy_one(bool forward, size_t smem, int* blocks_per_sm);
inline size_t uneven_smem_bytes(int land_max, int work_max)
{
    return 128 + (size_t)(2LL * land_max + work_max) * sizeof(float2);
}

// Row stride (elements) of a tile's work rows (rows are not padded inside):
// at least L, and chosen so that the 16 threads of a half-warp never meet on
// one bank of 8-byte words across rows.  A stage that maps consecutive
// threads to consecutive lines (the strided sides of four-step jobs) puts
// H = 16/T positions of each of T lines in a half-warp; a stage that maps
// them along a line puts H = G = 256/T positions of each of 16/G lines there
// (short lines, G < 16).  Rows then start H * (odd) banks apart when
// stride mod 2H == H.  (A tile of 32 strided lines has both kinds of stage;
// its lines-fast stages win: H = 1.)  Padding inside the rows (i + i/16)
// bought no fewer shared-memory wavefronts on the batched-uneven mix once
// the rows are placed this way, and cost an address step per access.
inline int uneven_line_stride(long long L, long long T, bool cfast)
{
    const long long G = kUnevenThreads / T;
    long long H = 1;
    if (cfast && T <= 16) H = 16 / T;
    else if (!cfast && G < 16) H = G;
    long long ls = L;
    if (H < 16)
        while (ls % (2 * H) != H) ++ls;
    return (int)ls;
}

// Landing row stride of a contiguous-input tile (0: rows of L, first stage
// along a line).  Tiles of 2 to 8 lines land in rows H = 16/T banks apart
// (stride mod 2H == H, even, so the 16-byte copies stay aligned) and their
// first stage maps threads across lines: its radix-R groups would otherwise
// fill a half-warp at stride R (8-way for radix 8).
inline int uneven_land_row(long long L, long long T, bool in_tfast)
{
    if (in_tfast || T < 2 || T > 8) return 0;
    const long long H = 16 / T;
    long long lr = L;
    while (lr % (2 * H) != H) ++lr;
    return (int)lr;
}

}  // namespace fbfft
