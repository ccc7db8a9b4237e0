// fb_internal.h -- declarations shared by the library's translation units.
// Not part of the public ABI (that is include/fb_fft.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace fbfft {

constexpr int kMaxStages = 8;
constexpr int kElemsPerThread = 16;  // E: complex values one thread holds per stage
constexpr int kGenericElems = 8;     // E of the generic (run-time schedule) kernel

// Thread-block shapes of the line-pass kernels (tile capacity = compute
// threads x values per thread): power-of-two lines take compile-time kernels
// of 64, 128, 256 or 512 compute threads (fft_p2.cuh); lines with a factor 3
// or 5 take the mixed kernels (up to 2048 points) or the generic kernel, which
// reads its whole schedule at run time.
constexpr int kGenericThreads = 512;  // generic kernel: 512 x 8 = 4096 values per tile
// Mixed kernels (power-of-two radices at compile time, then 5s and 3s):
// 256 threads x 8 values, lines up to 2048 with a factor 3 or 5.
constexpr int kMixedThreads = 256;
constexpr int kMixedElems = 8;
constexpr int kMixedMaxLen = kMixedThreads * kMixedElems;
constexpr int kMaxLineLog2 = 12;  // 4096

// One kernel launch of the line pass: 1-D DFTs of length L along one axis of a
// strided view.  Line (o, c) starts at o*so + c*sc; its element n sits n*sn
// further on (separate strides for input and output).  A CTA takes a tile of
// T = 2^logT consecutive c at one o.
struct PassDesc {
    const float2* in;
    float2* out;
    const float2* tw;      // twiddle buffer; stage s table at tw + twoff[s]
    const float2* ptw_lo;  // four-step post-twiddle, exp(-2 pi i m / ptw_n) for m < 2^ptw_log
    const float2* ptw_hi;  // exp(-2 pi i (m << ptw_log) / ptw_n)
    long long in_sn, in_sc, in_so;
    long long out_sk, out_sc, out_so;
    long long C;           // lines per outer index o
    long long tiles_per_o; // ceil(C / T)
    long long ntiles;      // O * tiles_per_o
    int L;                 // line length
    int LS;                // shared-memory line stride (elements, padded)
    int logT;              // T = 1 << logT lines per tile
    int nst;               // number of Stockham stages
    int radix[kMaxStages];
    int ns[kMaxStages];    // product of the radices before stage s
    int twoff[kMaxStages]; // element offset of stage s's twiddle table
    unsigned ns_mag[kMaxStages];  // ceil(2^32 / ns[s]) for ns[s] > 1: j mod ns[s] by one multiply-high
    int in_tfast;          // 1: first stage maps threads across lines (input contiguous across c)
    int out_tfast;         // 1: last stage maps threads across lines (output contiguous across c)
    int ptw;               // 1: multiply output (c, k) by exp(s 2 pi i c k / ptw_n)
    int ptw_log;
    int apply_scale;
    float scale;
    int async_io;          // 1: tiles move by TMA (bulk / tensor copies), double-buffered
    int land_stride;       // elements between the two landing buffers (multiple of 16)
    int box_rows;          // rows per 3-D TMA box (a divisor of L, <= 256)
    int* err;              // device error word: 1 = a bounded wait gave up
    unsigned debug_extra_tx;  // test hook: bytes announced per tile that never arrive
    int tws;               // stage-twiddle entries the kernel copies to shared memory
    int ptw_smem;          // 1: the kernel copies the four-step tables (ptw_lo, ptw_hi) to shared memory
    int ptw_hi_cnt;        // entries of ptw_hi (ptw_lo has 2^ptw_log)
    int evict_first;       // 1: tile loads of `in` take the L2 evict-first policy (the caller's input, read once)
    int evict_last;        // 1: tile stores take the L2 evict-last policy (read again by the next pass)
    // Batched uneven lengths: element offset of each transform's start in
    // in / out (device arrays, or null for the regular strides above).
    // Contiguous layouts index them by line, strided ones by outer index.
    const long long* off_in;
    const long long* off_out;
    // Batched-uneven job tables (k_fft_uneven): which exec buffer `in` and
    // `out` refer to (0 the caller's input, 1 its output, 2 the plan's
    // scratch; the pointer fields then hold element offsets into it), or 3:
    // the pointer fields are the addresses themselves.
    int in_buf;
    int out_buf;
    // k_fft_uneven, contiguous input: 0 = lines land as rows of L and the
    // first stage maps threads along a line; > 0 = rows of land_row elements
    // and the first stage maps threads across lines (tiles of 2 to 8 lines).
    int land_row;
    // Batched uneven lengths in one launch (k_fft_uneven_one): dependency
    // slot s + 1 whose finished-tile counter this job's tiles raise (four-step
    // columns), or that it waits for (four-step rows) until the counter
    // reaches dep_need; 0 = none.
    int dep_post;
    int dep;
    int dep_need;
};

// Fill ns[] (product of the earlier radices) and its multiply-high
// reciprocals from radix[0..nst).  floor(j * ceil(2^32/x) / 2^32) == j / x
// while j * x < 2^32, which holds for every j < L / radix the kernels use.
inline void set_stage_products(PassDesc& d)
{
    long long Ns = 1;
    for (int s = 0; s < d.nst; ++s) {
        d.ns[s] = (int)Ns;
        d.ns_mag[s] = Ns > 1 ? (unsigned)(((1ULL << 32) + (unsigned long long)Ns - 1) / (unsigned long long)Ns) : 0u;
        Ns *= d.radix[s];
    }
}

// Several passes of one mixed kernel in one launch (batched uneven lengths:
// every length with the same power-of-two factor).  Job j owns global tiles
// [tile_start[j], tile_start[j+1]); its descriptor is d[j] (plain copies, no
// TMA: the jobs' tiles go through offset tables).  The whole struct is the
// kernel parameter (about 20 KB, under the 32 KB parameter limit), so a
// captured graph holds it by value.
constexpr int kMultiMax = 64;
struct MultiArgs {
    long long tile_start[kMultiMax + 1];
    int njobs;
    int land_max;  // elements of a landing buffer; two of them, then two work buffers
    int work_max;  // elements of a work buffer
    PassDesc d[kMultiMax];
};
cudaError_t mixed_multi_launch(bool forward, int lg2, const MultiArgs& a, long long grid, size_t smem,
                               cudaStream_t stream);
cudaError_t mixed_multi_occupancy(bool forward, int lg2, size_t smem, int* blocks_per_sm);

// Kernel argument: the descriptor plus the TMA tensor maps of the c-fast
// input/output views {C, L, O} (encoded per launch, they hold addresses).
struct LineArgs {
    PassDesc d;
    CUtensorMap tm_in;
    CUtensorMap tm_out;
};

// Shared memory (bytes) the line pass needs for a tile of T lines of length L:
// alignment slack and mbarriers (256 B), one or two dense landing buffers and the
// padded work buffer.
inline long long land_stride_elems(int L, int T) { return ((long long)L * T + 15) & ~15LL; }
inline size_t line_smem_bytes(long long land_elems, int L, int T, int nst, bool async, int tws = 0)
{
    const long long land = land_elems * (async ? 2 : 1);
    const long long LS = (long long)L + (L >> 4) + 16;  // bound on every mode's work-row stride
    const long long work = nst <= 1 ? 0 : LS * T;
    return 256 + (size_t)(land + work + tws) * sizeof(float2);  // alignment slack + mbarriers
}

// One compiled line-pass kernel.  kind 0: compile-time power-of-two kernel
// (lg = log2 L, io = its IoMode); 1: generic kernel; 2: mixed kernel
// (lg = log2 of L's power-of-two factor); 3: plane pass (lg1 = log2 rows,
// lg = log2 row length, launched in clusters of `cluster` CTAs).
struct LineKernel {
    void (*fn)(LineArgs);
    int threads;
    bool fwd;
    int lg;
    int io;
    int kind = 0;
    bool tc = false;     // radix-16 stages on the tensor cores
    int producers = 0;   // threads beside the compute threads (power-of-two kernels: producer warp(s))
    int split_regs = 0;  // > 0: registers per thread the kernel must be launched with (it
                         // rebalances them with setmaxnreg, which needs exactly that pool)
    int lg1 = 0;         // plane pass (kind 3): log2 of the rows per plane (lg: of the row length)
    int cluster = 0;     // > 1: CTAs per thread-block cluster
};
// Extra shared memory of a tensor-core line pass: B^T (4 KB) + alignment.
constexpr size_t kTcExtraSmem = 4096 + 128;
// The kernel for a pass; fn == nullptr when that combination is not compiled.
LineKernel line_kernel_p2(int threads, bool forward, int lg, int io);
// Tensor-core variant (power-of-two L >= 256, the thread count the planner
// picks for that length and layout).
LineKernel line_kernel_p2tc(int threads, bool forward, int lg, int io);
LineKernel line_kernel_generic(bool forward);
// Plane pass (fft_plane.cuh): 2-D DFT over L1 = 2^lg1 rows of L2 = 2^lg2
// contiguous values, one cluster of CTAs per plane; lg1, lg2 in {7, 8};
// threads = compute threads per CTA, 512 or 256 (not for 256 x 256).
LineKernel line_kernel_plane(bool forward, int lg1, int lg2, int threads);
long long plane_smem_bytes(int lg1, int lg2, int threads);
// Clusters of a cluster kernel that fit the GPU at once.
cudaError_t line_cluster_occupancy(const LineKernel& k, size_t smem, int* clusters);
LineKernel line_kernel_mixed(bool forward, int lg2);
// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum,
// once per (kernel, device); split_regs > 0 also checks the kernel's register
// count (see LineKernel::split_regs).
cudaError_t kernel_smem_optin(const void* fn, int split_regs);
// Launch / occupancy / name of a table entry (shared-memory opt-in handled inside).
cudaError_t line_launch(const LineKernel& k, const LineArgs& a, long long grid, size_t smem, cudaStream_t stream);
cudaError_t line_occupancy(const LineKernel& k, size_t smem, int* blocks_per_sm);
void line_kernel_name(const LineKernel& k, char* buf, size_t n);

// Twiddle table jobs: K0 evaluates exp(-2 pi i m / D) in FP64 and rounds to FP32.
//   kind 0 (linear): entry i has m = (i * mult) mod D
//   kind 1 (stage):  entry i = (r-1)*Ns + k has m = r*k, D = Ns*R
struct TwiddleJob {
    long long offset;
    long long count;
    long long D;
    long long mult;
    int kind;
    int R;
    int Ns;
};
cudaError_t launch_twiddles(float2* tw, const TwiddleJob& job, cudaStream_t stream);

}  // namespace fbfft
