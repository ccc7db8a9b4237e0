// fb_fft.cu -- host side of the FFT function block: planner, plan object and
// the C ABI declared in include/fb_fft.h.
//
// Schedules (all passes are launches of the Stockham line-pass kernel):
//   rank 1, N <= 4096    one pass, lines contiguous.
//   rank 1, N  > 4096    "four-step" N = N1*N2, n = N2*n1 + n2, k = k1 + N1*k2:
//                        pass A: length-N1 DFTs down the N2 columns, output
//                                multiplied by exp(s*2*pi*i*n2*k1/N)  (-> scratch)
//                        pass B: length-N2 DFTs along the N1 rows, written
//                                transposed to X[k1 + N1*k2]          (-> out)
//                        The batch runs in chunks of at most 512 MiB of
//                        intermediate: few, long launches keep every CTA's
//                        TMA pipeline full (measured faster than chunks small
//                        enough to keep the intermediate in the 126 MB L2).
//   rank 2/3             one pass per axis (last axis first), in place on out.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <cudaTypedefs.h>

#include "fb_fft.h"
#include "fb_host.h"
#include "fb_internal.h"
#include "fb_plan.h"
#include "fft_p2.cuh"
#include "fft_uneven.cuh"

using namespace fbfft;
using namespace fbfft::plan;

namespace {

std::atomic<long long> g_launches{0};
thread_local char g_last_error[256] = "";

// Record a failed CUDA call (readable through fb_fft_last_error) and map it.
int cuda_fail(cudaError_t e, const char* what)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    cudaGetLastError();  // clear a non-sticky error so later launch checks do not see it
    return FB_FFT_ERR_CUDA;
}
#define FB_CK(call)                                      \
    do {                                                 \
        cudaError_t fb_e_ = (call);                      \
        if (fb_e_ != cudaSuccess) return cuda_fail(fb_e_, #call); \
    } while (0)
constexpr uint32_t kMagic = 0xFBFF7A11u;
constexpr uint32_t kDead = 0xDEADFBFFu;

// Four-step batch chunk: bytes of intermediate (scratch) per column/row pass pair.
long long fourstep_chunk_bytes()
{
    static long long v = [] {
        const char* s = std::getenv("FB_FFT_FOURSTEP_CHUNK_BYTES");
        long long b = s ? std::atoll(s) : 0;
        return b > 0 ? b : (512LL << 20);
    }();
    return v;
}

// Side streams of a batched-uneven plan (independent length groups overlap).
int many_streams()
{
    static int v = [] {
        const char* s = std::getenv("FB_FFT_MANY_STREAMS");
        const int n = s ? std::atoi(s) : 0;
        return n >= 1 && n <= 32 ? n : 4;
    }();
    return v;
}

// Batched-uneven plans: mixed-kernel passes of one phase and power-of-two
// factor, run as one k_fft_mixed_multi launch.
struct MultiLaunch {
    std::vector<int> members;  // pass indices
    int lg2 = 0;
    int phase = 0;             // 0: single passes and four-step columns, 1: four-step rows
    int slot = 0;
    long long tiles = 0;
    long long grid = 0;
    int land_max = 0;
    int work_max = 0;
    size_t smem = 0;
};

struct TwiddleBuilder {
    std::vector<TwiddleJob> jobs;
    long long total = 0;
    struct Cached {
        long long L;
        std::vector<int> radix;
        std::vector<int> off;
    };
    std::vector<Cached> stage_cache;  // (L, radix schedule) -> offsets

    long long add_linear(long long count, long long D, long long mult)
    {
        TwiddleJob j{total, count, D, mult, 0, 0, 0};
        jobs.push_back(j);
        const long long off = total;
        total += (count + 1) & ~1LL;  // keep every table 16-byte aligned
        return off;
    }
    // Stage tables of length L; returns offsets per stage, then (entry nst)
    // the 16 x 15 factor table of a split last stage (p2_tw_split), else 0.
    std::vector<int> add_stages(long long L, const int* radix, int nst)
    {
        const std::vector<int> key(radix, radix + nst);
        for (auto& e : stage_cache)
            if (e.L == L && e.radix == key) return e.off;
        std::vector<int> off(nst + 1, 0);
        TwiddleJob js[kMaxStages + 1];
        int nj = 0;
        total += stage_tables(L, radix, nst, total, js, &nj, off.data());
        jobs.insert(jobs.end(), js, js + nj);
        stage_cache.push_back({L, key, off});
        return off;
    }
    // the interface make_line_pass takes (tables in a growing buffer: always room)
    bool stages(long long L, const int* radix, int nst, int* off)
    {
        const std::vector<int> v = add_stages(L, radix, nst);
        for (int s = 0; s <= nst; ++s) off[s] = v[s];
        return true;
    }
};

// Plane pass: the 2-D DFT over `planes` contiguous planes of L1 rows x L2
// values (the two trailing axes of a multi-D transform, one cluster per plane).
int make_plane_pass(PassPlan& p, TwiddleBuilder& twb, long long L1, long long L2, long long planes)
{
    p = PassPlan{};
    PassDesc& d = p.d;
    p.kind = 3;
    p.io = -1;
    p.lg = ilog2ll(L2);
    p.lg1 = ilog2ll(L1);
    // compute threads per CTA: FB_FFT_PLANE_THREADS = 256 or 512 picks one
    // where both are compiled
    p.threads = 512;
    if (const char* s = std::getenv("FB_FFT_PLANE_THREADS"))
        if (std::atoi(s) == 256 && line_kernel_plane(true, p.lg1, p.lg, 256).fn) p.threads = 256;
    const LineKernel k = line_kernel_plane(true, p.lg1, p.lg, p.threads);
    if (!k.fn || (L1 & (L1 - 1)) || (L2 & (L2 - 1))) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    // second-stage tables of the two-stage schedules (radix 16, then L / 16),
    // the same the line passes of these lengths use: [0] rows, [1] columns
    for (int side = 0; side < 2; ++side) {
        const long long L = side == 0 ? L2 : L1;
        int radix[kMaxStages];
        const int nst = factorize(L, radix, kMaxStages);
        if (nst != 2 || radix[0] != 16 || radix[1] != L / 16) return FB_FFT_ERR_UNSUPPORTED_SIZE;
        d.twoff[side] = twb.add_stages(L, radix, nst)[1];
    }
    d.L = (int)L2;
    d.in_sn = L2, d.in_so = L1 * L2;
    d.out_sk = L2, d.out_so = L1 * L2;
    d.C = L2;
    d.tiles_per_o = 1;
    d.ntiles = planes;
    d.scale = 1.0f;
    p.async_ok = planes < (1LL << 31);
    p.smem = (size_t)plane_smem_bytes(p.lg1, p.lg, p.threads);
    p.grid = planes * k.cluster;  // capped to the clusters that fit when the plan is built
    return FB_FFT_OK;
}

}  // namespace

struct fb_fft_plan_s {
    uint32_t magic = kMagic;
    int device = 0;
    int rank = 0;
    long long dims[3] = {1, 1, 1};
    long long batch = 0;
    unsigned flags = 0;
    cudaStream_t stream = nullptr;
    long long N = 1;
    std::vector<PassPlan> passes;
    std::vector<const char*> group_names;
    float2* tw = nullptr;
    long long tw_elems = 0;
    float2* scratch = nullptr;
    size_t scratch_bytes = 0;
    bool ext_scratch = false;  // scratch supplied per exec (server plans)
    float2* staging = nullptr;
    size_t staging_bytes = 0;
    // fb_fft_exec_host on pinned arrays: the batch in chunks, each chunk's
    // copy in, transform and copy out on three streams so they overlap
    fb_fft_plan_s* host_chunk = nullptr;  // plan of host_chunk_batch transforms
    fb_fft_plan_s* host_tail = nullptr;   // plan of the last, shorter chunk
    long long host_chunk_batch = 0;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    std::vector<cudaEvent_t> host_ev;
    int* err = nullptr;  // device error word written by bounded waits
    long long smem_len_max = 0;
    bool debug_timeout = false;  // test hook: make every TMA wait run out
    bool no_plane = false;       // plane passes disabled (their cluster does not fit this GPU)
    bool no_evict_first = false; // FB_FFT_EVICT_FIRST=0: first-pass loads without the L2 evict-first policy
    bool no_evict_last = false;  // FB_FFT_EVICT_LAST=0: intermediate stores without the L2 evict-last policy
    long long l2_bytes = 0;      // the device's L2 size
    // batched uneven lengths (fb_fft_plan_many)
    bool many = false;
    long long total = 0;                 // elements of the packed layout
    std::vector<long long> lengths, offsets;
    long long* d_off = nullptr;          // device offset tables of all passes
    std::vector<long long> h_off;        // host copy, uploaded once
    int nslots = 1;
    std::vector<cudaStream_t> side;      // side streams (slots)
    cudaStream_t capture = nullptr;      // where graphs are captured (the caller's may be uncapturable)
    std::vector<cudaEvent_t> fork_join;  // [0] fork, [1 + s] join of slot s
    bool use_graph = true;
    long long chunk_bytes = 0;   // 0: fourstep_chunk_bytes()
    bool odd_first = false;
    int max_lines = 0;
    bool merge_mixed = true;               // batched uneven: merged mixed-kernel launches
    // batched uneven, one-kernel engine: every pass is a job of phase 0 (single
    // passes and four-step columns) or phase 1 (four-step rows), one launch of
    // k_fft_uneven each (engine 2), or both in the one launch below; jobs and
    // tile prefixes in device tables
    bool uneven = false;
    struct UnevenPhase {
        std::vector<int> jobs;   // pass indices
        long long tiles = 0;
        long long grid = 0;
        int land_max = 16, work_max = 16;
        size_t smem = 0;
        PassDesc* d_jobs = nullptr;
        int* d_tiles = nullptr;
    };
    UnevenPhase uphase[2];
    // one launch per exec (k_fft_uneven_one, the default): both phases' jobs
    // in one table (phase 0, then phase 1), four-step rows waiting on their
    // chunk's columns through device counters
    bool uneven_one = false;
    int uneven_slots = 0;                  // dependency slots: one per four-step chunk
    UnevenPhase uone;                      // the merged table's jobs, tiles, grid, shared memory
    unsigned long long* d_sync = nullptr;  // [2 + uneven_slots] counters, zero between execs
    void* d_uneven = nullptr;              // one allocation: job and tile tables, counters
    std::vector<MultiLaunch> multis;
    std::unique_ptr<MultiArgs> margs;      // launch-argument staging (copied at every launch)
    struct GraphEntry {
        const void* in;
        void* out;
        int dir;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    // profiling
    bool profiling = false;
    std::vector<cudaEvent_t> ev;  // pairs
    std::vector<int> ev_group;
    size_t ev_used = 0;
};

namespace {

bool plan_ok(fb_fft_plan_t p) { return p && p->magic == kMagic; }

void free_plan(fb_fft_plan_s* p)
{
    if (!p) return;
    free_plan(p->host_chunk);
    free_plan(p->host_tail);
    if (p->h2d) cudaStreamDestroy(p->h2d);
    if (p->d2h) cudaStreamDestroy(p->d2h);
    for (cudaEvent_t e : p->host_ev) cudaEventDestroy(e);
    if (p->tw) cudaFree(p->tw);
    if (p->scratch) cudaFree(p->scratch);
    if (p->staging) cudaFree(p->staging);
    if (p->err) cudaFree(p->err);
    if (p->d_off) cudaFree(p->d_off);
    if (p->d_uneven) cudaFree(p->d_uneven);
    for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
    for (cudaStream_t st : p->side) cudaStreamDestroy(st);
    if (p->capture) cudaStreamDestroy(p->capture);
    for (cudaEvent_t e : p->fork_join) cudaEventDestroy(e);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    p->magic = kDead;
    delete p;
}

// Packed layout of a batch of uneven 1-D transforms: transform i starts at
// offsets[i] = sum over j < i of lengths[j] rounded up to even, so every
// transform starts 16-byte aligned (a TMA requirement).
long long many_layout(int count, const long long* lengths, long long* offsets)
{
    long long off = 0;
    for (int i = 0; i < count; ++i) {
        if (offsets) offsets[i] = off;
        off += (lengths[i] + 1) & ~1LL;
    }
    return off;
}

// Whether a batched-uneven plan runs on the one-kernel engine: the default
// (engine 0: one launch per exec; engine 2: one launch per phase) unless one
// launch per length is asked for, and every length either fits one job
// (<= 2048 points) or splits into two that do.
bool use_uneven_engine(int count, const long long* lengths, const fb_fft_many_opts* opts)
{
    if (opts && ((opts->engine != 0 && opts->engine != 2) || opts->per_length != 0)) return false;
    for (int i = 0; i < count; ++i) {
        const long long L = lengths[i];
        if (L <= kUnevenMaxLen) continue;
        long long best = 0;
        for (long long d = 1; d * d <= L; ++d)
            if (L % d == 0 && L / d <= kUnevenMaxLen) best = d;
        if (best == 0) return false;
    }
    return true;
}

// Radix schedule of a line of the one-kernel batched-uneven engine
// (k_fft_uneven): the power-of-two part as radix-8 stages and one radix-4 or
// radix-2 stage, then the 5s, then the 3s -- the order of kinds the kernel
// runs its middle stages in.  The kernel has no one-stage form, so a
// schedule of a single radix ends with a radix-1 stage (a copy).  Returns the
// stage count.
int uneven_factorize(long long L, int* r)
{
    int c = 0, a = 0;
    long long n = L;
    while (n % 2 == 0) n /= 2, ++a;
    for (int i = 0; i < a / 3; ++i) r[c++] = 8;
    if (a % 3 == 2) r[c++] = 4;
    if (a % 3 == 1) r[c++] = 2;
    while (n % 5 == 0) n /= 5, r[c++] = 5;
    while (n % 3 == 0) n /= 3, r[c++] = 3;
    while (c < 2) r[c++] = 1;
    return c;
}

// Lines per tile of a job of L-point lines (C per outer index) on the
// one-kernel engine: as many as fit 2048 values, a power of two, at most 32
// where a side is strided (rows of T consecutive values), at most C rounded up.
long long uneven_tile_lines(long long L, long long C, bool cfast)
{
    long long T = pow2floor(kUnevenCap / L);
    T = std::min<long long>(T, cfast ? 32 : kUnevenThreads);
    return std::max<long long>(1, std::min(T, pow2ceil(C)));
}

// One job of the one-kernel engine: L-point DFTs over lines (o, c), strides in
// elements (offsets into the exec buffers are set by the caller); tiles of T
// lines, T L <= 2048 values.
int make_uneven_pass(PassPlan& p, TwiddleBuilder& twb, long long L, long long O, long long C, long long in_sn,
                     long long in_sc, long long in_so, long long out_sk, long long out_sc, long long out_so,
                     bool in_tfast, bool out_tfast, bool ptw)
{
    p = PassPlan{};
    PassDesc& d = p.d;
    if (L < 1 || L > kUnevenMaxLen || !is_smooth(L)) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    p.kind = 4;
    p.io = -1;
    p.threads = kUnevenThreads;
    d.nst = uneven_factorize(L, d.radix);
    set_stage_products(d);
    const std::vector<int> off = twb.add_stages(L, d.radix, d.nst);
    for (int s = 0; s < d.nst; ++s) d.twoff[s] = off[s];
    const bool cfast = in_tfast || out_tfast;
    const long long T = uneven_tile_lines(L, C, cfast);
    d.L = (int)L;
    d.LS = uneven_line_stride(L, T, cfast);
    d.logT = ilog2ll(T);
    d.in_sn = in_sn, d.in_sc = in_sc, d.in_so = in_so;
    d.out_sk = out_sk, d.out_sc = out_sc, d.out_so = out_so;
    d.C = C;
    d.tiles_per_o = (C + T - 1) / T;
    d.ntiles = O * d.tiles_per_o;
    d.in_tfast = in_tfast ? 1 : 0;
    d.out_tfast = out_tfast ? 1 : 0;
    d.ptw = ptw ? 1 : 0;
    d.scale = 1.0f;
    d.land_row = uneven_land_row(L, T, in_tfast);
    d.land_stride = (int)(((d.land_row ? d.land_row : L) * T + 15) & ~15LL);
    p.async_ok = false;
    const int padded = (int)(((long long)d.LS * T + 15) & ~15LL);
    p.smem = uneven_smem_bytes(std::max(d.land_stride, padded), padded);
    p.grid = 0;  // launched through its phase's launch only
    return FB_FFT_OK;
}

// Issue cost of one tile in k_fft_uneven, in values handled per thread: per
// stage, the butterfly rounds a thread runs (radix R values each) plus a
// fixed stage overhead, plus the tile's load and store.  A tile of T lines
// has 256 / T threads per line; the cost hardly depends on how full the tile
// is, so lengths whose tiles stay half empty cost twice per value.
long long uneven_tile_cost(long long L, long long T)
{
    int r[kMaxStages];
    const int nst = uneven_factorize(L, r);
    const long long G = kUnevenThreads / T;
    long long c = 10;
    for (int s = 0; s < nst; ++s) {
        const long long LR = L / r[s];
        c += (LR + G - 1) / G * r[s] + 6;
    }
    return c;
}

// The four-step split of n > 2048 on the one-kernel engine: n = n1 * n2 (the
// column and row lengths), both at most 2048.  Among all such pairs, the one
// whose two jobs cost the fewest tile issues per transform (above), keeping
// the strided rows at least as long as the split with the largest n1 <= sqrt(n)
// has them (up to 8 values): on 4096 lengths in [64, 65536] this cut the
// modelled issue cost by 7 %.
int split_uneven(long long n, long long* n1, long long* n2)
{
    long long base = 0;
    for (long long d = 1; d * d <= n; ++d)
        if (n % d == 0 && n / d <= kUnevenMaxLen) base = d;
    if (base == 0) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    auto seg = [&](long long a) {  // shorter strided row of the pair (a, n / a)
        const long long b = n / a;
        return std::min(uneven_tile_lines(a, b, true), uneven_tile_lines(b, a, true));
    };
    auto cost = [&](long long a) {
        const long long b = n / a, ta = uneven_tile_lines(a, b, true), tb = uneven_tile_lines(b, a, true);
        return (b + ta - 1) / ta * uneven_tile_cost(a, ta) + (a + tb - 1) / tb * uneven_tile_cost(b, tb);
    };
    const long long min_seg = std::min<long long>(8, seg(base));
    long long best = base, best_cost = cost(base);
    for (long long a = 1; a <= kUnevenMaxLen && a <= n; ++a) {
        if (n % a || n / a > kUnevenMaxLen || seg(a) < min_seg) continue;
        const long long c = cost(a);
        if (c < best_cost) best = a, best_cost = c;
    }
    *n1 = best, *n2 = n / best;
    return FB_FFT_OK;
}

// Batched uneven lengths on the one-kernel engine: every distinct length is
// one job over all its transforms (offset tables), or, above 2048 points, a
// four-step pair of jobs per chunk of transforms, each chunk with its own
// scratch region.  Phase 0 holds single passes and four-step columns, phase
// 1 the four-step rows; the default plan runs both in one launch of
// k_fft_uneven_one (each row chunk after its columns, through a dependency
// slot per chunk), engine 2 each phase as one launch of k_fft_uneven.
int schedule_uneven(fb_fft_plan_s* p, TwiddleBuilder& twb)
{
    std::vector<std::pair<long long, std::vector<long long>>> groups;  // (L, transform indices)
    {
        std::vector<long long> order(p->lengths.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (long long)i;
        std::stable_sort(order.begin(), order.end(),
                         [&](long long a, long long b) { return p->lengths[a] > p->lengths[b]; });
        for (long long i : order) {
            if (groups.empty() || groups.back().first != p->lengths[i]) groups.push_back({p->lengths[i], {}});
            groups.back().second.push_back(i);
        }
    }
    if (p->uneven_one)
        p->group_names = {"many.uneven"};
    else
        p->group_names = {"many.uneven.phase0", "many.uneven.phase1"};
    long long scratch_need = 0;
    for (auto& g : groups) {
        const long long L = g.first;
        const std::vector<long long>& idx = g.second;
        auto push_offsets = [&](size_t b0, size_t nb) {
            const long long at = (long long)p->h_off.size();
            for (size_t k = b0; k < b0 + nb; ++k) p->h_off.push_back(p->offsets[idx[k]]);
            return at;
        };
        if (L <= kUnevenMaxLen) {
            PassPlan q;
            int rc = make_uneven_pass(q, twb, L, 1, (long long)idx.size(), 1, L, 0, 1, L, 0, false, false, false);
            if (rc != FB_FFT_OK) return rc;
            q.off_in_idx = q.off_out_idx = push_offsets(0, idx.size());
            q.src = kBufIn, q.dst = kBufOut;
            q.group = 0;
            q.last = true;
            q.scale_n = L;
            p->passes.push_back(q);
            p->smem_len_max = std::max(p->smem_len_max, L);
            continue;
        }
        long long N1, N2;
        int rc = split_uneven(L, &N1, &N2);
        if (rc != FB_FFT_OK) return rc;
        const int plog = (ilog2ll(L) + 1) / 2;
        const long long lo_cnt = 1LL << plog, hi_cnt = (L + lo_cnt - 1) >> plog;
        const long long lo_off = twb.add_linear(lo_cnt, L, 1);
        const long long hi_off = twb.add_linear(hi_cnt, L, lo_cnt);
        const long long cnt = (long long)idx.size();
        const long long cbytes = p->chunk_bytes > 0 ? p->chunk_bytes : fourstep_chunk_bytes();
        const long long chunk = std::max(1LL, std::min(cnt, cbytes / (L * 8)));
        for (long long b0 = 0; b0 < cnt; b0 += chunk) {
            const long long nb = std::min(chunk, cnt - b0);
            const long long at = push_offsets((size_t)b0, (size_t)nb);
            const long long region = scratch_need;
            scratch_need += (nb * L + 31) & ~31LL;  // keep regions 256-byte aligned
            PassPlan a, r;
            rc = make_uneven_pass(a, twb, N1, nb, N2, N2, 1, L, N2, 1, L, true, true, true);
            if (rc != FB_FFT_OK) return rc;
            a.d.ptw_log = plog;
            a.d.ptw_lo = reinterpret_cast<const float2*>(lo_off);
            a.d.ptw_hi = reinterpret_cast<const float2*>(hi_off);
            a.off_in_idx = at;
            a.src = kBufIn, a.dst = kBufScratch, a.dst_off = region;
            a.group = 0;
            rc = make_uneven_pass(r, twb, N2, nb, N1, 1, N2, L, N1, 1, L, false, true, false);
            if (rc != FB_FFT_OK) return rc;
            r.off_out_idx = at;
            r.src = kBufScratch, r.src_off = region, r.dst = kBufOut;
            r.group = 1;
            r.last = true;
            r.scale_n = L;
            // one launch: the rows of this chunk wait for all its column tiles
            const int slot = p->uneven_slots++;
            a.d.dep_post = slot + 1;
            r.d.dep = slot + 1;
            if (a.d.ntiles >= (1LL << 31)) return FB_FFT_ERR_UNSUPPORTED_SIZE;
            r.d.dep_need = (int)a.d.ntiles;
            p->passes.push_back(a);
            p->passes.push_back(r);
        }
        p->smem_len_max = std::max(p->smem_len_max, std::max(N1, N2));
    }
    for (int i = 0; i < (int)p->passes.size(); ++i) {
        PassPlan& q = p->passes[i];
        fb_fft_plan_s::UnevenPhase& ph = p->uphase[q.group];
        ph.jobs.push_back(i);
        ph.tiles += q.d.ntiles;
        const int padded = (int)(((long long)q.d.LS * (1LL << q.d.logT) + 15) & ~15LL);
        ph.land_max = std::max(ph.land_max, std::max(q.d.land_stride, padded));  // also a work buffer
        ph.work_max = std::max(ph.work_max, padded);
    }
    for (auto& ph : p->uphase) ph.smem = uneven_smem_bytes(ph.land_max, ph.work_max);
    fb_fft_plan_s::UnevenPhase& one = p->uone;
    for (const fb_fft_plan_s::UnevenPhase& ph : p->uphase) {
        one.jobs.insert(one.jobs.end(), ph.jobs.begin(), ph.jobs.end());
        one.tiles += ph.tiles;
        one.land_max = std::max(one.land_max, ph.land_max);
        one.work_max = std::max(one.work_max, ph.work_max);
    }
    one.smem = uneven_smem_bytes(one.land_max, one.work_max);
    p->scratch_bytes = (size_t)scratch_need * sizeof(float2);
    p->tw_elems = std::max(2LL, twb.total);
    return FB_FFT_OK;
}

// Batched uneven lengths: one pass (or one four-step pair per chunk) per
// distinct length, each covering all transforms of that length through an
// offset table.  Without merging, single-pass groups are spread over side
// streams 1..nslots-1 and four-step groups over all slots, each slot with its
// own scratch region; with merging (the default), mixed-kernel passes become
// merged launches and every four-step chunk has its own scratch region.
int schedule_many(fb_fft_plan_s* p, TwiddleBuilder& twb)
{
    std::vector<std::pair<long long, std::vector<long long>>> groups;  // (L, transform indices)
    {
        std::vector<long long> order(p->lengths.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = (long long)i;
        std::stable_sort(order.begin(), order.end(),
                         [&](long long a, long long b) { return p->lengths[a] > p->lengths[b]; });
        for (long long i : order) {
            if (groups.empty() || groups.back().first != p->lengths[i]) groups.push_back({p->lengths[i], {}});
            groups.back().second.push_back(i);
        }
    }
    p->group_names = {"many.single_pass", "many.fourstep.columns", "many.fourstep.rows", "many.merged_mixed"};
    // every slot owns a scratch region, so four-step groups on different
    // slots overlap; groups on one slot reuse its region in turn
    std::vector<long long> slot_need(p->nslots, 0);
    int rr = 0, rr4 = 0;
    for (auto& g : groups) {
        const long long L = g.first;
        const std::vector<long long>& idx = g.second;
        const bool pow2 = (L & (L - 1)) == 0;
        auto push_offsets = [&](size_t b0, size_t nb) {
            const long long at = (long long)p->h_off.size();
            for (size_t k = b0; k < b0 + nb; ++k) p->h_off.push_back(p->offsets[idx[k]]);
            return at;
        };
        // with merged launches, lengths that only the generic (run-time
        // schedule) kernel would take run as two mixed passes (four-step) in
        // the merged launches instead
        const bool via_fourstep = p->merge_mixed && !pow2 && L > kMixedMaxLen;
        if (L <= FB_FFT_MAX_SMEM_LEN && !via_fourstep) {
            PassPlan q;
            int rc = make_line_pass(q, twb, L, 1, (long long)idx.size(), 1, L, 0, 1, L, 0, false, false, false,
                                    p->odd_first, p->max_lines);
            if (rc != FB_FFT_OK) return rc;
            q.off_in_idx = q.off_out_idx = push_offsets(0, idx.size());
            if (!pow2) q.async_ok = false;  // the generic kernel copies offset-table tiles itself
            q.src = kBufIn, q.dst = kBufOut;
            q.group = 0;
            q.last = true;
            q.scale_n = L;
            q.slot = p->nslots > 1 ? 1 + (rr++ % (p->nslots - 1)) : 0;
            p->passes.push_back(q);
            p->smem_len_max = std::max(p->smem_len_max, L);
            continue;
        }
        long long N1, N2;
        int rc = L <= FB_FFT_MAX_SMEM_LEN ? split_square(L, &N1, &N2) : split_fourstep(L, &N1, &N2);
        if (rc != FB_FFT_OK) return rc;
        const int plog = (ilog2ll(L) + 1) / 2;
        const long long lo_cnt = 1LL << plog, hi_cnt = (L + lo_cnt - 1) >> plog;
        const long long lo_off = twb.add_linear(lo_cnt, L, 1);
        const long long hi_off = twb.add_linear(hi_cnt, L, lo_cnt);
        const long long cnt = (long long)idx.size();
        const long long cbytes = p->chunk_bytes > 0 ? p->chunk_bytes : fourstep_chunk_bytes();
        const long long chunk = std::max(1LL, std::min(cnt, cbytes / (L * 8)));
        const int slot = rr4++ % p->nslots;
        slot_need[slot] = std::max(slot_need[slot], chunk * L);
        for (long long b0 = 0; b0 < cnt; b0 += chunk) {
            const long long nb = std::min(chunk, cnt - b0);
            const long long at = push_offsets((size_t)b0, (size_t)nb);
            PassPlan a, r;
            rc = make_line_pass(a, twb, N1, nb, N2, N2, 1, L, N2, 1, L, true, true, true, p->odd_first, p->max_lines);
            if (rc != FB_FFT_OK) return rc;
            a.d.ptw_log = plog;
            a.d.ptw_lo = reinterpret_cast<const float2*>(lo_off);
            a.d.ptw_hi = reinterpret_cast<const float2*>(hi_off);
            ptw_to_smem(a, hi_cnt);
            a.off_in_idx = at;
            if ((N1 & (N1 - 1)) != 0) a.async_ok = false;
            a.src = kBufIn, a.dst = kBufScratch;
            a.group = 1;
            a.slot = slot;
            rc = make_line_pass(r, twb, N2, nb, N1, 1, N2, L, N1, 1, L, false, true, false, p->odd_first,
                                p->max_lines);
            if (rc != FB_FFT_OK) return rc;
            r.off_out_idx = at;
            if ((N2 & (N2 - 1)) != 0) r.async_ok = false;
            r.src = kBufScratch, r.dst = kBufOut;
            r.group = 2;
            r.last = true;
            r.scale_n = L;
            r.slot = slot;
            p->passes.push_back(a);
            p->passes.push_back(r);
        }
        p->smem_len_max = std::max(p->smem_len_max, std::max(N1, N2));
    }
    long long scratch_need = 0;
    if (!p->merge_mixed) {
        // scratch regions: slot s starts after the regions of slots < s
        std::vector<long long> region(p->nslots, 0);
        for (int sl = 0; sl < p->nslots; ++sl) {
            region[sl] = scratch_need;
            scratch_need += (slot_need[sl] + 31) & ~31LL;  // keep regions 256-byte aligned
        }
        for (PassPlan& q : p->passes) {
            if (q.dst == kBufScratch) q.dst_off = region[q.slot];
            if (q.src == kBufScratch) q.src_off = region[q.slot];
        }
    } else {
        // every four-step chunk its own region: a merged launch runs many
        // chunks' column (or row) passes at once.  Passes were pushed as
        // (columns, rows) pairs, so a row pass takes its column pass's region.
        long long last = 0;
        for (PassPlan& q : p->passes) {
            if (q.dst == kBufScratch) {
                const long long O = q.d.ntiles / q.d.tiles_per_o;
                last = scratch_need;
                q.dst_off = last;
                scratch_need += (O * (long long)q.d.L * q.d.C + 31) & ~31LL;
            }
            if (q.src == kBufScratch) q.src_off = last;
        }
        // merged launches: mixed-kernel passes grouped by phase and power-of-two factor
        std::map<std::pair<int, int>, std::vector<int>> buckets;
        for (int i = 0; i < (int)p->passes.size(); ++i) {
            const PassPlan& q = p->passes[i];
            if (q.kind == 2) buckets[{q.group == 2 ? 1 : 0, q.lg}].push_back(i);
        }
        int rrm = 0;
        for (auto& kv : buckets) {
            const std::vector<int>& v = kv.second;
            if (v.size() < 2) continue;
            for (size_t b0 = 0; b0 < v.size(); b0 += kMultiMax) {
                MultiLaunch m;
                m.phase = kv.first.first;
                m.lg2 = kv.first.second;
                m.slot = rrm++ % p->nslots;
                long long work_max = 0;
                for (size_t k = b0; k < std::min(v.size(), b0 + (size_t)kMultiMax); ++k) {
                    PassPlan& q = p->passes[v[k]];
                    q.multi = (int)p->multis.size();
                    m.members.push_back(v[k]);
                    m.tiles += q.d.ntiles;
                    m.land_max = std::max(m.land_max, q.d.land_stride);
                    work_max = std::max(work_max, ((long long)q.d.L + (q.d.L >> 4) + 16) << q.d.logT);
                }
                m.work_max = (int)((work_max + 15) & ~15LL);
                m.smem = 256 + (size_t)(2LL * m.land_max + 2LL * m.work_max) * sizeof(float2);
                p->multis.push_back(m);
            }
        }
    }
    p->scratch_bytes = (size_t)scratch_need * sizeof(float2);
    p->tw_elems = std::max(2LL, twb.total);
    return FB_FFT_OK;
}

// Kernel launches one exec of a plan makes.
long long launches_per_exec(const fb_fft_plan_s* p)
{
    if (p->uneven && p->uneven_one) return p->uone.jobs.empty() ? 0 : 1;
    if (p->uneven) return (p->uphase[0].jobs.empty() ? 0 : 1) + (p->uphase[1].jobs.empty() ? 0 : 1);
    long long n = (long long)p->multis.size();
    for (const PassPlan& q : p->passes) n += q.multi < 0 ? 1 : 0;
    return n;
}

// Invariants of a schedule, checked on the host before anything launches:
// offset tables only on the caller's buffers (never on the scratch), table
// ranges inside the offset buffer, slots inside the plan's side streams.
int check_schedule(const fb_fft_plan_s* p)
{
    const long long nofs = (long long)p->h_off.size();
    for (const PassPlan& q : p->passes) {
        const long long O = q.d.tiles_per_o ? q.d.ntiles / q.d.tiles_per_o : 0;
        if (q.off_in_idx >= 0) {
            const long long need = q.d.in_tfast ? O : q.d.C;  // strided: per outer index, contiguous: per line
            if (q.src != kBufIn || q.off_in_idx + need > nofs) return FB_FFT_ERR_INVALID_ARG;
        }
        if (q.off_out_idx >= 0) {
            const long long need = q.d.out_tfast ? O : q.d.C;
            if (q.dst != kBufOut || q.off_out_idx + need > nofs) return FB_FFT_ERR_INVALID_ARG;
        }
        if (!p->many && (q.off_in_idx >= 0 || q.off_out_idx >= 0)) return FB_FFT_ERR_INVALID_ARG;
        // a four-step pass's scratch window (O transforms of L*C values) lies inside the scratch
        const long long scratch_elems = (long long)(p->scratch_bytes / sizeof(float2));
        const long long window = O * (long long)q.d.L * q.d.C;
        if (q.dst == kBufScratch && q.dst_off + window > scratch_elems) return FB_FFT_ERR_INVALID_ARG;
        if (q.src == kBufScratch && q.src_off + window > scratch_elems) return FB_FFT_ERR_INVALID_ARG;
        if (q.slot < 0 || q.slot >= p->nslots) return FB_FFT_ERR_INVALID_ARG;
        if (q.multi >= (int)p->multis.size()) return FB_FFT_ERR_INVALID_ARG;
    }
    // merged launches: members are mixed-kernel passes of the launch's phase
    // and factor, at most kMultiMax of them, with landing tiles that fit
    for (const MultiLaunch& m : p->multis) {
        if (m.members.empty() || m.members.size() > (size_t)kMultiMax) return FB_FFT_ERR_INVALID_ARG;
        if (m.slot < 0 || m.slot >= p->nslots || m.smem > kMaxSmemBytes) return FB_FFT_ERR_INVALID_ARG;
        for (int i : m.members) {
            const PassPlan& q = p->passes[i];
            if (q.kind != 2 || q.lg != m.lg2 || (q.group == 2 ? 1 : 0) != m.phase) return FB_FFT_ERR_INVALID_ARG;
            if (q.d.land_stride > m.land_max || ((long long)q.d.L << q.d.logT) > m.land_max)
                return FB_FFT_ERR_INVALID_ARG;
        }
    }
    return FB_FFT_OK;
}

// Rank-2/3 plans: run the two trailing axes as one plane pass when
// FB_FFT_PLANE=1 and the plane shape is compiled (128 or 256 by 128 or 256).
// Off by default: on the 256 x 256 x 128 volume the plane pass takes 68 us
// where the two line passes it replaces take 47 us (its cluster-wide phases
// leave one CTA per SM waiting at every barrier).
bool use_plane_pass(const fb_fft_plan_s* p)
{
    if (p->rank < 2 || p->no_plane || (p->flags & FB_FFT_TENSOR_CORES)) return false;
    const long long L1 = p->dims[p->rank - 2], L2 = p->dims[p->rank - 1];
    if (!line_kernel_plane(true, ilog2ll(L1), ilog2ll(L2), 512).fn) return false;
    long long planes = p->batch;
    for (int e = 0; e < p->rank - 2; ++e) planes *= p->dims[e];
    if (planes < 1 || planes >= (1LL << 31)) return false;
    const char* s = std::getenv("FB_FFT_PLANE");
    return s && s[0] == '1';
}

// Host part of planning: the pass list and the twiddle jobs (no device work).
int schedule_plan(fb_fft_plan_s* p, TwiddleBuilder& twb)
{
    if (p->many) {
        const int rc = p->uneven ? schedule_uneven(p, twb) : schedule_many(p, twb);
        return rc != FB_FFT_OK ? rc : check_schedule(p);
    }
    const long long B = p->batch;
    const bool tc = (p->flags & FB_FFT_TENSOR_CORES) != 0;
    if (p->rank == 1 && p->N > FB_FFT_MAX_SMEM_LEN) {
        long long N1, N2;
        int rc = split_fourstep(p->N, &N1, &N2);
        if (rc != FB_FFT_OK) return rc;
        const long long N = p->N;
        const int plog = (ilog2ll(N) + 1) / 2;  // split 2^plog >= sqrt(N)
        const long long lo_cnt = 1LL << plog;
        const long long hi_cnt = (N + lo_cnt - 1) >> plog;
        const long long lo_off = twb.add_linear(lo_cnt, N, 1);
        const long long hi_off = twb.add_linear(hi_cnt, N, lo_cnt);
        const long long chunk = std::max(1LL, std::min(B, fourstep_chunk_bytes() / (N * 8)));
        p->scratch_bytes = (size_t)(chunk * N) * sizeof(float2);
        p->group_names = {"fourstep.columns", "fourstep.rows"};
        for (long long b0 = 0; b0 < B; b0 += chunk) {
            const long long nb = std::min(chunk, B - b0);
            PassPlan a, r;
            rc = make_line_pass(a, twb, N1, nb, N2, N2, 1, N, N2, 1, N, true, true, true, false, 0, tc);
            if (rc != FB_FFT_OK) return rc;
            a.d.ptw_log = plog;
            ptw_to_smem(a, hi_cnt);
            a.src = kBufIn, a.src_off = b0 * N;
            a.dst = kBufScratch, a.dst_off = 0;
            a.group = 0;
            // stash table offsets in the pointer fields until exec binds them
            a.d.ptw_lo = reinterpret_cast<const float2*>(lo_off);
            a.d.ptw_hi = reinterpret_cast<const float2*>(hi_off);
            rc = make_line_pass(r, twb, N2, nb, N1, 1, N2, N, N1, 1, N, false, true, false, false, 0, tc);
            if (rc != FB_FFT_OK) return rc;
            r.src = kBufScratch, r.src_off = 0;
            r.dst = kBufOut, r.dst_off = b0 * N;
            r.group = 1;
            r.last = true;
            p->passes.push_back(a);
            p->passes.push_back(r);
        }
        p->smem_len_max = std::max(N1, N2);
    } else {
        static const char* axis_names[3] = {"axis0", "axis1", "axis2"};
        static const char* one_name[1] = {"lines"};
        bool first = true;
        int ngroups = 0;
        int ax_top = p->rank - 1;
        if (use_plane_pass(p)) {  // the two trailing axes in one pass
            const long long L1 = p->dims[p->rank - 2], L2 = p->dims[p->rank - 1];
            long long planes = B;
            for (int e = 0; e < p->rank - 2; ++e) planes *= p->dims[e];
            PassPlan q;
            const int rc = make_plane_pass(q, twb, L1, L2, planes);
            if (rc != FB_FFT_OK) return rc;
            q.src = kBufIn;
            q.dst = kBufOut;
            q.group = ngroups++;
            first = false;
            p->passes.push_back(q);
            p->group_names.push_back("plane");
            p->smem_len_max = std::max(L1, L2);
            ax_top = p->rank - 3;
        }
        for (int ax = ax_top; ax >= 0; --ax) {
            const long long L = p->dims[ax];
            if (L == 1) continue;
            long long S = 1, Opre = 1;
            for (int e = ax + 1; e < p->rank; ++e) S *= p->dims[e];
            for (int e = 0; e < ax; ++e) Opre *= p->dims[e];
            PassPlan q;
            int rc;
            if (S == 1)
                rc = make_line_pass(q, twb, L, 1, B * Opre, 1, L, 0, 1, L, 0, false, false, false, false, 0, tc);
            else
                rc = make_line_pass(q, twb, L, B * Opre, S, S, 1, L * S, S, 1, L * S, true, true, false, false, 0,
                                    tc);
            if (rc != FB_FFT_OK) return rc;
            q.src = first ? kBufIn : kBufOut;
            q.dst = kBufOut;
            q.group = ngroups++;
            first = false;
            p->passes.push_back(q);
            p->group_names.push_back(p->rank == 1 ? one_name[0] : axis_names[ax]);
            p->smem_len_max = std::max(p->smem_len_max, L);
        }
        if (!p->passes.empty()) p->passes.back().last = true;
    }
    p->tw_elems = std::max(2LL, twb.total);
    return check_schedule(p);
}

int build_plan(fb_fft_plan_s* p)
{
    TwiddleBuilder twb;
    int rc = schedule_plan(p, twb);
    if (rc != FB_FFT_OK) return rc;
    // a plane pass needs one whole cluster resident; where none fits, plan
    // the axis passes instead
    for (const PassPlan& q : p->passes) {
        if (q.kind != 3) continue;
        int ncl = 0;
        if (line_cluster_occupancy(pass_kernel(q, true), q.smem, &ncl) != cudaSuccess || ncl < 1) {
            cudaGetLastError();
            p->no_plane = true;
        }
    }
    if (p->no_plane) {
        p->passes.clear();
        p->group_names.clear();
        p->smem_len_max = 0;
        twb = TwiddleBuilder();
        rc = schedule_plan(p, twb);
        if (rc != FB_FFT_OK) return rc;
    }
    // Twiddle tables: one device buffer, built by the FP64 kernel.
    if (cudaMalloc(&p->tw, (size_t)p->tw_elems * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        p->tw = nullptr;
        return FB_FFT_ERR_ALLOC;
    }
    for (const TwiddleJob& j : twb.jobs) FB_CK(launch_twiddles(p->tw, j, p->stream));
    if (cudaMalloc(&p->err, 16 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        p->err = nullptr;
        return FB_FFT_ERR_ALLOC;
    }
    FB_CK(cudaMemsetAsync(p->err, 0, 16 * sizeof(int), p->stream));
    int sms = 0;
    FB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    for (PassPlan& q : p->passes) {
        int occ = 0;
        const LineKernel k = pass_kernel(q, true);
        if (q.kind == 4) {  // batched-uneven job: bound into its phase's table below
            q.d.err = p->err;
            q.d.tw = p->tw;
            if (q.d.ptw) {
                q.d.ptw_lo = p->tw + reinterpret_cast<long long>(q.d.ptw_lo);
                q.d.ptw_hi = p->tw + reinterpret_cast<long long>(q.d.ptw_hi);
            }
            continue;
        }
        if (q.kind == 3) {  // persistent clusters: as many as fit at once
            int ncl = 0;
            FB_CK(line_cluster_occupancy(k, q.smem, &ncl));
            q.grid = std::min(q.grid, (long long)ncl * k.cluster);
            q.d.err = p->err;
            q.d.tw = p->tw;
            continue;
        }
        FB_CK(line_occupancy(k, q.smem, &occ));
        if (occ < 1) return cuda_fail(cudaErrorInvalidConfiguration, "line pass occupancy");
        // The occupancy query answers one CTA per SM for every kernel that
        // uses the tensor cores; two fit (shared memory, registers, 2 x 64 of
        // 512 TMEM columns) and measured 1.36x faster, so size those grids from
        // the resources.  (A grid above what fits would only run in waves.)
        if (q.tc) occ = std::max(occ, pass_ctas_per_sm(q, q.smem));
        q.grid = std::min(q.grid, (long long)sms * occ);
        q.d.err = p->err;
        q.d.tw = p->tw;
        if (q.d.ptw) {
            q.d.ptw_lo = p->tw + reinterpret_cast<long long>(q.d.ptw_lo);
            q.d.ptw_hi = p->tw + reinterpret_cast<long long>(q.d.ptw_hi);
        }
    }
    if (p->scratch_bytes && !p->ext_scratch) {
        if (cudaMalloc(&p->scratch, p->scratch_bytes) != cudaSuccess) {
            cudaGetLastError();
            p->scratch = nullptr;
            return FB_FFT_ERR_ALLOC;
        }
    }
    if (p->many) {
        if (!p->h_off.empty()) {
            if (cudaMalloc(&p->d_off, p->h_off.size() * sizeof(long long)) != cudaSuccess) {
                cudaGetLastError();
                p->d_off = nullptr;
                return FB_FFT_ERR_ALLOC;
            }
            FB_CK(cudaMemcpyAsync(p->d_off, p->h_off.data(), p->h_off.size() * sizeof(long long),
                                  cudaMemcpyHostToDevice, p->stream));
        }
        for (PassPlan& q : p->passes) {
            if (q.off_in_idx >= 0) q.d.off_in = p->d_off + q.off_in_idx;
            if (q.off_out_idx >= 0) q.d.off_out = p->d_off + q.off_out_idx;
        }
        if (p->uneven) {
            // job tables: descriptors with buffer kinds and element offsets in
            // place of the exec's pointers, and tile prefixes -- each phase's,
            // and both phases' for the one-launch form -- and that form's
            // counters, in one device allocation
            std::vector<PassDesc> jobs;
            std::vector<int> tiles;
            fb_fft_plan_s::UnevenPhase* tabs[3] = {&p->uphase[0], &p->uphase[1], &p->uone};
            size_t job_at[3], tile_at[3];
            for (int ph = 0; ph < 3; ++ph) {
                fb_fft_plan_s::UnevenPhase& u = *tabs[ph];
                job_at[ph] = jobs.size();
                tile_at[ph] = tiles.size();
                long long t = 0;
                for (int i : u.jobs) {
                    const PassPlan& q = p->passes[i];
                    PassDesc d = q.d;
                    d.in = reinterpret_cast<const float2*>(static_cast<uintptr_t>(q.src_off));
                    d.in_buf = q.src == kBufIn ? 0 : (q.src == kBufOut ? 1 : 2);
                    d.out = reinterpret_cast<float2*>(static_cast<uintptr_t>(q.dst_off));
                    d.out_buf = q.dst == kBufOut ? 1 : 2;
                    d.apply_scale = q.last ? 1 : 0;
                    d.scale = (float)(1.0 / (double)(q.scale_n ? q.scale_n : 1));
                    jobs.push_back(d);
                    tiles.push_back((int)t);
                    t += q.d.ntiles;
                }
                if (t >= (1LL << 31)) return FB_FFT_ERR_UNSUPPORTED_SIZE;
                tiles.push_back((int)t);
            }
            const size_t jb = jobs.size() * sizeof(PassDesc), tb = tiles.size() * sizeof(int);
            const size_t sb_at = (jb + tb + 15) & ~(size_t)15;
            const int nsync = 2 + p->uneven_slots;
            const size_t sb = (size_t)nsync * sizeof(unsigned long long);
            if (cudaMalloc(&p->d_uneven, sb_at + sb) != cudaSuccess) {
                cudaGetLastError();
                p->d_uneven = nullptr;
                return FB_FFT_ERR_ALLOC;
            }
            PassDesc* dj = static_cast<PassDesc*>(p->d_uneven);
            int* dt = reinterpret_cast<int*>(static_cast<char*>(p->d_uneven) + jb);
            p->d_sync = reinterpret_cast<unsigned long long*>(static_cast<char*>(p->d_uneven) + sb_at);
            if (jb) FB_CK(cudaMemcpyAsync(dj, jobs.data(), jb, cudaMemcpyHostToDevice, p->stream));
            FB_CK(cudaMemcpyAsync(dt, tiles.data(), tb, cudaMemcpyHostToDevice, p->stream));
            FB_CK(cudaMemsetAsync(p->d_sync, 0, sb, p->stream));
            for (int ph = 0; ph < 3; ++ph) {
                fb_fft_plan_s::UnevenPhase& u = *tabs[ph];
                u.d_jobs = dj + job_at[ph];
                u.d_tiles = dt + tile_at[ph];
                if (u.jobs.empty()) continue;
                int occ = 0;
                if (ph == 2)
                    FB_CK(uneven_occupancy_one(true, u.smem, &occ));
                else
                    FB_CK(uneven_occupancy(true, u.smem, &occ));
                if (occ < 1) return cuda_fail(cudaErrorInvalidConfiguration, "uneven pass occupancy");
                u.grid = std::min(u.tiles, (long long)sms * occ);
            }
        }
        for (MultiLaunch& m : p->multis) {
            int occ = 0;
            FB_CK(mixed_multi_occupancy(true, m.lg2, m.smem, &occ));
            if (occ < 1) return cuda_fail(cudaErrorInvalidConfiguration, "merged pass occupancy");
            m.grid = std::min(m.tiles, (long long)sms * occ);
            for (int i : m.members) p->passes[i].grid = 0;  // launched through the merged launch only
        }
        if (!p->multis.empty()) {
            p->margs.reset(new (std::nothrow) MultiArgs());
            if (!p->margs) return FB_FFT_ERR_ALLOC;
        }
        for (int sl = 0; sl < p->nslots; ++sl) {
            cudaStream_t st;
            FB_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            p->side.push_back(st);
        }
        FB_CK(cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking));
        // [0] fork, [1 + s] join of slot s, [1 + nslots + s] end of phase 0 on slot s
        for (int e = 0; e <= 2 * p->nslots; ++e) {
            cudaEvent_t ev;
            FB_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            p->fork_join.push_back(ev);
        }
    }
    FB_CK(cudaStreamSynchronize(p->stream));
    return FB_FFT_OK;
}

// Launch one pass of a plan on `stream` (profiling events, when on, go on
// the same stream).
int launch_pass(fb_fft_plan_s* p, const PassPlan& q, const float2* in, float2* out, bool fwd, cudaStream_t stream,
                bool count, float2* scratch, int* err)
{
    const float2* src = q.src == kBufIn ? in : (q.src == kBufOut ? out : scratch);
    float2* dst = q.dst == kBufOut ? out : scratch;
    LineArgs args;
    const size_t smem = line_args(args, q, src + q.src_off, dst + q.dst_off, err);
    PassDesc& d = args.d;
    d.evict_first = (q.src == kBufIn && in != out && !p->many && !p->no_evict_first) ? 1 : 0;
    // a pass whose output the next pass reads keeps it in L2 when it fits
    // with room to spare (the caller's input, loaded evict-first, and other
    // work share the cache); the last pass stores with the default policy, so
    // nothing stays favoured after the exec
    const long long out_bytes = (long long)q.d.L * q.d.C * (q.d.ntiles / std::max(1LL, q.d.tiles_per_o)) * 8;
    d.evict_last = (!q.last && !p->many && !p->no_evict_last && out_bytes * 10 <= p->l2_bytes * 6) ? 1 : 0;
    if (p->debug_timeout && d.async_io) d.debug_extra_tx = 16;
    if (q.last && !fwd && (p->flags & FB_FFT_SCALE_INV_N)) {
        d.apply_scale = 1;
        d.scale = (float)(1.0 / (double)(q.scale_n ? q.scale_n : p->N));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (p->profiling) {
        if (p->ev_used + 2 > p->ev.size()) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                FB_CK(cudaEventCreate(&e));
                p->ev.push_back(e);
            }
            p->ev_group.resize(p->ev.size() / 2, 0);
        }
        e0 = p->ev[p->ev_used];
        e1 = p->ev[p->ev_used + 1];
        p->ev_group[p->ev_used / 2] = q.group;
        p->ev_used += 2;
        cudaEventRecord(e0, stream);
    }
    const LineKernel k = pass_kernel(q, fwd);
    const cudaError_t le = line_launch(k, args, q.grid, smem, stream);
    if (le != cudaSuccess) {
        char nm[64];
        line_kernel_name(k, nm, sizeof(nm));
        return cuda_fail(le, nm);
    }
    if (count) g_launches.fetch_add(1, std::memory_order_relaxed);
    if (p->profiling) cudaEventRecord(e1, stream);
    return FB_FFT_OK;
}

// One merged launch of mixed-kernel passes (MultiArgs by value).
int launch_multi(fb_fft_plan_s* p, const MultiLaunch& m, const float2* in, float2* out, bool fwd,
                 cudaStream_t stream, bool count)
{
    MultiArgs& a = *p->margs;
    a.njobs = (int)m.members.size();
    a.land_max = m.land_max;
    a.work_max = m.work_max;
    a.tile_start[0] = 0;
    for (int k = 0; k < a.njobs; ++k) {
        const PassPlan& q = p->passes[m.members[k]];
        PassDesc d = q.d;
        const float2* src = q.src == kBufIn ? in : (q.src == kBufOut ? out : p->scratch);
        float2* dst = q.dst == kBufOut ? out : p->scratch;
        d.in = src + q.src_off;
        d.out = dst + q.dst_off;
        d.async_io = 0;
        if (q.last && !fwd && (p->flags & FB_FFT_SCALE_INV_N)) {
            d.apply_scale = 1;
            d.scale = (float)(1.0 / (double)(q.scale_n ? q.scale_n : p->N));
        }
        a.d[k] = d;
        a.tile_start[k + 1] = a.tile_start[k] + d.ntiles;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (p->profiling) {
        if (p->ev_used + 2 > p->ev.size()) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                FB_CK(cudaEventCreate(&e));
                p->ev.push_back(e);
            }
            p->ev_group.resize(p->ev.size() / 2, 0);
        }
        e0 = p->ev[p->ev_used];
        e1 = p->ev[p->ev_used + 1];
        p->ev_group[p->ev_used / 2] = 3;
        p->ev_used += 2;
        cudaEventRecord(e0, stream);
    }
    const cudaError_t le = mixed_multi_launch(fwd, m.lg2, a, m.grid, m.smem, stream);
    if (le != cudaSuccess) return cuda_fail(le, "k_fft_mixed_multi");
    if (count) g_launches.fetch_add(1, std::memory_order_relaxed);
    if (p->profiling) cudaEventRecord(e1, stream);
    return FB_FFT_OK;
}

// Batched uneven plan: fork the side streams off `origin`, run each pass on
// its slot, join back into `origin`.  With merged launches: phase 0 (single
// passes, four-step columns), every slot waits for every slot, phase 1
// (four-step rows).
int launch_many(fb_fft_plan_s* p, cudaStream_t origin, const float2* in, float2* out, bool fwd, bool count)
{
    FB_CK(cudaEventRecord(p->fork_join[0], origin));
    for (int sl = 0; sl < p->nslots; ++sl) FB_CK(cudaStreamWaitEvent(p->side[sl], p->fork_join[0], 0));
    if (!p->merge_mixed) {
        for (const PassPlan& q : p->passes) {
            const int rc = launch_pass(p, q, in, out, fwd, p->side[q.slot], count, p->scratch, nullptr);
            if (rc != FB_FFT_OK) return rc;
        }
    } else {
        for (int phase = 0; phase < 2; ++phase) {
            if (phase == 1) {
                for (int sl = 0; sl < p->nslots; ++sl)
                    FB_CK(cudaEventRecord(p->fork_join[1 + p->nslots + sl], p->side[sl]));
                for (int sl = 0; sl < p->nslots; ++sl)
                    for (int s2 = 0; s2 < p->nslots; ++s2)
                        if (s2 != sl) FB_CK(cudaStreamWaitEvent(p->side[sl], p->fork_join[1 + p->nslots + s2], 0));
            }
            for (const MultiLaunch& m : p->multis) {
                if (m.phase != phase) continue;
                const int rc = launch_multi(p, m, in, out, fwd, p->side[m.slot], count);
                if (rc != FB_FFT_OK) return rc;
            }
            for (const PassPlan& q : p->passes) {
                if (q.multi >= 0 || (q.group == 2 ? 1 : 0) != phase) continue;
                const int rc = launch_pass(p, q, in, out, fwd, p->side[q.slot], count, p->scratch, nullptr);
                if (rc != FB_FFT_OK) return rc;
            }
        }
    }
    for (int sl = 0; sl < p->nslots; ++sl) {
        FB_CK(cudaEventRecord(p->fork_join[1 + sl], p->side[sl]));
        FB_CK(cudaStreamWaitEvent(origin, p->fork_join[1 + sl], 0));
    }
    return FB_FFT_OK;
}

// Batched uneven plan on the one-kernel engine: one launch of every pass
// (k_fft_uneven_one), or phase 0 (single passes, four-step columns) then
// phase 1 (four-step rows), one launch each.
int launch_uneven(fb_fft_plan_s* p, cudaStream_t stream, const float2* in, float2* out, bool fwd, bool count)
{
    const bool one = p->uneven_one;
    for (int ph = 0; ph < (one ? 1 : 2); ++ph) {
        const fb_fft_plan_s::UnevenPhase& u = one ? p->uone : p->uphase[ph];
        if (u.jobs.empty()) continue;
        UnevenArgs a{};
        a.jobs = u.d_jobs;
        a.tile_start = u.d_tiles;
        a.in = in;
        a.out = out;
        a.scratch = p->scratch;
        a.njobs = (int)u.jobs.size();
        a.land_max = u.land_max;
        a.work_max = u.work_max;
        a.scale_on = (!fwd && (p->flags & FB_FFT_SCALE_INV_N)) ? 1 : 0;
        a.sync = p->d_sync;
        a.nsync = 2 + p->uneven_slots;
        a.dep_extra = p->debug_timeout ? (1 << 30) : 0;
        cudaEvent_t e1 = nullptr;
        if (p->profiling) {
            if (p->ev_used + 2 > p->ev.size()) {
                for (int i = 0; i < 64; ++i) {
                    cudaEvent_t e;
                    FB_CK(cudaEventCreate(&e));
                    p->ev.push_back(e);
                }
                p->ev_group.resize(p->ev.size() / 2, 0);
            }
            e1 = p->ev[p->ev_used + 1];
            p->ev_group[p->ev_used / 2] = ph;
            cudaEventRecord(p->ev[p->ev_used], stream);
            p->ev_used += 2;
        }
        const cudaError_t le =
            one ? uneven_launch_one(fwd, a, u.grid, u.smem, stream) : uneven_launch(fwd, a, u.grid, u.smem, stream);
        if (le != cudaSuccess) return cuda_fail(le, one ? "k_fft_uneven_one" : "k_fft_uneven");
        if (count) g_launches.fetch_add(1, std::memory_order_relaxed);
        if (e1) cudaEventRecord(e1, stream);
    }
    return FB_FFT_OK;
}

// Batched uneven plan, replayed as one CUDA graph per (in, out, direction):
// the first exec with a new triple captures its launch sequence (the
// one-kernel engine's single launch, or the fork/join sequence of engine 1).
int exec_many(fb_fft_plan_s* p, const float2* in, float2* out, int direction)
{
    const bool fwd = direction == FB_FFT_FORWARD;
    auto launch_all = [&](cudaStream_t st, bool count) {
        return p->uneven ? launch_uneven(p, st, in, out, fwd, count) : launch_many(p, st, in, out, fwd, count);
    };
    if (!p->use_graph || p->profiling || p->debug_timeout || (p->uneven && !p->uneven_one))
        return launch_all(p->stream, true);
    for (auto& g : p->graphs)
        if (g.in == in && g.out == out && g.dir == direction) {
            FB_CK(cudaGraphLaunch(g.exec, p->stream));
            g_launches.fetch_add(launches_per_exec(p), std::memory_order_relaxed);
            return FB_FFT_OK;
        }
    // capture on the plan's own stream (the caller's may be the legacy
    // default stream, which cannot be captured), launch on the caller's
    FB_CK(cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal));
    const int rc = launch_all(p->capture, false);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(p->capture, &graph);
    if (rc != FB_FFT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
    if (p->graphs.size() >= 8) {  // keep the most recent few
        cudaGraphExecDestroy(p->graphs.front().exec);
        p->graphs.erase(p->graphs.begin());
    }
    p->graphs.push_back({in, out, direction, exec});
    FB_CK(cudaGraphLaunch(exec, p->stream));
    g_launches.fetch_add(launches_per_exec(p), std::memory_order_relaxed);
    return FB_FFT_OK;
}

int tc_pass_count(const std::vector<PassPlan>& passes)
{
    return (int)std::count_if(passes.begin(), passes.end(), [](const PassPlan& q) { return q.tc; });
}

long long plan_elems(const fb_fft_plan_s* p) { return p->many ? p->total : p->N * p->batch; }

int validate(int rank, const long long* dims, long long batch, unsigned flags, long long* N_out)
{
    if (rank < 1 || rank > 3 || !dims || batch < 0 || (flags & ~(FB_FFT_SCALE_INV_N | FB_FFT_TENSOR_CORES)))
        return FB_FFT_ERR_INVALID_ARG;
    long long N = 1;
    for (int d = 0; d < rank; ++d) {
        if (dims[d] < 1) return FB_FFT_ERR_INVALID_ARG;
        if (!is_smooth(dims[d])) return FB_FFT_ERR_UNSUPPORTED_SIZE;
        if (rank > 1 && dims[d] > FB_FFT_MAX_SMEM_LEN) return FB_FFT_ERR_UNSUPPORTED_SIZE;
        if (rank == 1 && dims[d] > FB_FFT_MAX_1D_LEN) return FB_FFT_ERR_UNSUPPORTED_SIZE;
        N *= dims[d];
    }
    if (batch > 0 && N > (1LL << 58) / batch) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    *N_out = N;
    return FB_FFT_OK;
}

// A regular plan's passes on `stream`, with the four-step intermediate in
// `scratch` and device-wait errors recorded in `err` (nullptr: the plan's).
int exec_lines(fb_fft_plan_s* p, const float2* in, float2* out, int direction, cudaStream_t stream, float2* scratch,
               int* err)
{
    const bool fwd = direction == FB_FFT_FORWARD;
    const size_t bytes = (size_t)(p->N * p->batch) * sizeof(float2);
    if (p->passes.empty()) {  // every axis has length 1: the DFT is the identity
        if (bytes && in != out) FB_CK(cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, stream));
        return FB_FFT_OK;
    }
    for (const PassPlan& q : p->passes) {
        const int rc = launch_pass(p, q, in, out, fwd, stream, true, scratch, err);
        if (rc != FB_FFT_OK) return rc;
    }
    return FB_FFT_OK;
}

int exec_device(fb_fft_plan_s* p, const float2* in, float2* out, int direction)
{
    if (p->many) return exec_many(p, in, out, direction);
    return exec_lines(p, in, out, direction, p->stream, p->scratch, nullptr);
}

// Plan construction shared by fb_fft_plan and the server; ext_scratch plans
// allocate no scratch (the caller passes one to exec_lines).
int plan_new(fb_fft_plan_s** out, int rank, const long long* dims, long long batch, unsigned flags,
             cudaStream_t stream, bool ext_scratch)
{
    *out = nullptr;
    long long N = 1;
    int rc0 = validate(rank, dims, batch, flags, &N);
    if (rc0 != FB_FFT_OK) return rc0;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return FB_FFT_ERR_NO_DEVICE;
    }
    fb_fft_plan_s* p = new (std::nothrow) fb_fft_plan_s();
    if (!p) return FB_FFT_ERR_ALLOC;
    cudaGetDevice(&p->device);
    p->rank = rank;
    for (int d = 0; d < rank; ++d) p->dims[d] = dims[d];
    p->batch = batch;
    p->flags = flags;
    p->stream = stream;
    p->N = N;
    p->ext_scratch = ext_scratch;
    if (const char* s = std::getenv("FB_FFT_EVICT_FIRST")) p->no_evict_first = s[0] == '0';
    if (const char* s = std::getenv("FB_FFT_EVICT_LAST")) p->no_evict_last = s[0] == '0';
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, p->device) != cudaSuccess) {
        cudaGetLastError();
        l2 = 0;
    }
    p->l2_bytes = l2;
    int rc = build_plan(p);
    if (rc != FB_FFT_OK) {
        free_plan(p);
        return rc;
    }
    *out = p;
    return FB_FFT_OK;
}

// fb_fft_exec_host pipelining: chunks of about this many bytes.
constexpr long long kHostChunkBytes = 32LL << 20;

bool host_pinned(const void* ptr)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

// Transforms per chunk for a pipelined host-array exec, or 0 when the call
// should run whole: batched regular plans of at least two chunks, pinned
// arrays (copies from pageable memory do not overlap), FB_FFT_HOST_PIPELINE
// not 0.  Chunks start 16-byte aligned (even count when N is odd), so they
// keep the TMA paths.
long long host_chunk_batch(const fb_fft_plan_s* p, const void* in, const void* out)
{
    if (p->many || p->batch < 2) return 0;
    const char* s = std::getenv("FB_FFT_HOST_PIPELINE");
    if (s && s[0] == '0') return 0;
    const long long item = p->N * (long long)sizeof(float2);
    long long cb = std::max(1LL, kHostChunkBytes / item);
    if (p->N % 2) cb = std::max(2LL, cb & ~1LL);
    cb = std::max(cb, (p->batch + 63) / 64);  // at most 64 chunks
    if (p->N % 2) cb = (cb + 1) & ~1LL;
    if (cb * 2 > p->batch) return 0;
    if (!host_pinned(in) || !host_pinned(out)) return 0;
    return cb;
}

// Copy in, transform and copy out chunk by chunk on the h2d stream, the
// plan's stream and the d2h stream: chunk k+1 arrives while chunk k is
// transformed and chunk k-1 leaves.  Each chunk runs a plan of its batch
// size (the same kernels and per-transform arithmetic as the whole plan).
int exec_host_pipelined(fb_fft_plan_s* p, const float2* hin, float2* hout, int direction, long long cb)
{
    const long long B = p->batch, N = p->N;
    const long long K = (B + cb - 1) / cb, tail = B - (K - 1) * cb;
    if (p->host_chunk_batch != cb) {
        free_plan(p->host_chunk);
        free_plan(p->host_tail);
        p->host_chunk = p->host_tail = nullptr;
        p->host_chunk_batch = 0;
        int rc = plan_new(&p->host_chunk, p->rank, p->dims, cb, p->flags, p->stream, false);
        if (rc != FB_FFT_OK) return rc;
        if (tail != cb) {
            rc = plan_new(&p->host_tail, p->rank, p->dims, tail, p->flags, p->stream, false);
            if (rc != FB_FFT_OK) return rc;
        }
        p->host_chunk_batch = cb;
    }
    if (!p->h2d) FB_CK(cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking));
    if (!p->d2h) FB_CK(cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking));
    while ((long long)p->host_ev.size() < 2 * K + 1) {
        cudaEvent_t e;
        FB_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p->host_ev.push_back(e);
    }
    auto enqueue = [&]() -> int {
        // the staging buffer is reused: start after the plan's earlier work
        FB_CK(cudaEventRecord(p->host_ev[2 * K], p->stream));
        FB_CK(cudaStreamWaitEvent(p->h2d, p->host_ev[2 * K], 0));
        for (long long k = 0; k < K; ++k) {
            const long long nb = k + 1 < K ? cb : tail;
            const long long off = k * cb * N;
            const size_t bytes = (size_t)(nb * N) * sizeof(float2);
            fb_fft_plan_s* c = nb == cb ? p->host_chunk : p->host_tail;
            FB_CK(cudaMemcpyAsync(p->staging + off, hin + off, bytes, cudaMemcpyHostToDevice, p->h2d));
            FB_CK(cudaEventRecord(p->host_ev[2 * k], p->h2d));
            FB_CK(cudaStreamWaitEvent(p->stream, p->host_ev[2 * k], 0));
            const int rc = exec_device(c, p->staging + off, p->staging + off, direction);
            if (rc != FB_FFT_OK) return rc;
            FB_CK(cudaEventRecord(p->host_ev[2 * k + 1], p->stream));
            FB_CK(cudaStreamWaitEvent(p->d2h, p->host_ev[2 * k + 1], 0));
            FB_CK(cudaMemcpyAsync(hout + off, p->staging + off, bytes, cudaMemcpyDeviceToHost, p->d2h));
        }
        return FB_FFT_OK;
    };
    int rc = enqueue();
    // wait for every copy, also after an error: the caller's arrays stay in use until then
    const cudaError_t e1 = cudaStreamSynchronize(p->h2d), e2 = cudaStreamSynchronize(p->stream),
                      e3 = cudaStreamSynchronize(p->d2h);
    if (rc != FB_FFT_OK) return rc;
    if (e1 != cudaSuccess) return cuda_fail(e1, "exec_host copy in");
    if (e2 != cudaSuccess) return cuda_fail(e2, "exec_host transform");
    if (e3 != cudaSuccess) return cuda_fail(e3, "exec_host copy out");
    rc = fb_fft_check(p->host_chunk);
    if (rc == FB_FFT_OK && p->host_tail) rc = fb_fft_check(p->host_tail);
    return rc;
}

}  // namespace

namespace fbfft {
namespace host {

int plan_create(fb_fft_plan_t* out, int rank, const long long* dims, long long batch, unsigned flags,
                cudaStream_t build_stream, bool ext_scratch)
{
    if (!out) return FB_FFT_ERR_INVALID_ARG;
    return plan_new(out, rank, dims, batch, flags, build_stream, ext_scratch);
}

long long plan_scratch_bytes(fb_fft_plan_t p) { return (long long)p->scratch_bytes; }

long long plan_table_bytes(fb_fft_plan_t p) { return p->tw_elems * (long long)sizeof(float2) + 16 * sizeof(int); }

long long plan_io_bytes(fb_fft_plan_t p) { return plan_elems(p) * (long long)sizeof(float2); }

int plan_exec_on(fb_fft_plan_t p, const void* in, void* out, int direction, cudaStream_t stream, void* scratch,
                 int* err)
{
    if (!plan_ok(p) || p->many) return FB_FFT_ERR_BAD_PLAN;
    if (p->scratch_bytes && !scratch && p->ext_scratch) return FB_FFT_ERR_INVALID_ARG;
    float2* s = p->ext_scratch ? (float2*)scratch : p->scratch;
    return exec_lines(p, (const float2*)in, (float2*)out, direction, stream, s, err);
}

void plan_free(fb_fft_plan_t p)
{
    if (plan_ok(p)) free_plan(p);
}

// The jobs of one request shape on the one-kernel engine, with the same
// pass geometry as a regular plan: a 1-D length up to 2048 is one job over
// the batch's lines; a longer one a four-step pair through the request's
// scratch (columns with the post-twiddle, then rows written transposed); a
// 2-D / 3-D shape one job per axis, last axis first, the first reading the
// input and the others in place on the output.
int recipe_create(BatchRecipe** out, int rank, const long long* dims, long long batch, unsigned flags,
                  cudaStream_t stream)
{
    if (!out) return FB_FFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (rank < 1 || rank > 3 || !dims || batch < 1) return FB_FFT_ERR_INVALID_ARG;
    if (flags & FB_FFT_TENSOR_CORES) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    long long N = 1;
    for (int e = 0; e < rank; ++e) {
        if (dims[e] < 1 || !is_smooth(dims[e])) return FB_FFT_ERR_UNSUPPORTED_SIZE;
        N *= dims[e];
    }
    if (N * batch >= (1LL << 40)) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    TwiddleBuilder twb;
    std::vector<PassPlan> passes;
    long long scratch = 0;
    int rc = FB_FFT_OK;
    if (rank == 1 && N > kUnevenMaxLen) {
        long long N1, N2;
        rc = split_uneven(N, &N1, &N2);
        if (rc != FB_FFT_OK) return rc;
        const int plog = (ilog2ll(N) + 1) / 2;
        const long long lo_cnt = 1LL << plog, hi_cnt = (N + lo_cnt - 1) >> plog;
        const long long lo_off = twb.add_linear(lo_cnt, N, 1);
        const long long hi_off = twb.add_linear(hi_cnt, N, lo_cnt);
        PassPlan a, r;
        rc = make_uneven_pass(a, twb, N1, batch, N2, N2, 1, N, N2, 1, N, true, true, true);
        if (rc != FB_FFT_OK) return rc;
        a.d.ptw_log = plog;
        a.d.ptw_lo = reinterpret_cast<const float2*>(lo_off);
        a.d.ptw_hi = reinterpret_cast<const float2*>(hi_off);
        a.src = kBufIn, a.dst = kBufScratch, a.group = 0;
        rc = make_uneven_pass(r, twb, N2, batch, N1, 1, N2, N, N1, 1, N, false, true, false);
        if (rc != FB_FFT_OK) return rc;
        r.src = kBufScratch, r.dst = kBufOut, r.group = 1, r.last = true;
        passes.push_back(a);
        passes.push_back(r);
        scratch = batch * N;
    } else {
        for (int ax = rank - 1; ax >= 0; --ax) {
            const long long L = dims[ax];
            if (L == 1 && !(ax == 0 && passes.empty())) continue;  // a shape of ones still copies
            long long S = 1, Opre = 1;
            for (int e = ax + 1; e < rank; ++e) S *= dims[e];
            for (int e = 0; e < ax; ++e) Opre *= dims[e];
            PassPlan q;
            if (S == 1 || L == 1)
                rc = make_uneven_pass(q, twb, L, 1, batch * N / L, 1, L, 0, 1, L, 0, false, false, false);
            else
                rc = make_uneven_pass(q, twb, L, batch * Opre, S, S, 1, L * S, S, 1, L * S, true, true, false);
            if (rc != FB_FFT_OK) return rc;
            q.src = passes.empty() ? kBufIn : kBufOut;
            q.dst = kBufOut;
            q.group = (int)passes.size();
            passes.push_back(q);
        }
        passes.back().last = true;
    }
    for (const PassPlan& q : passes)
        if (q.d.ntiles >= (1LL << 30)) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    BatchRecipe* r = new (std::nothrow) BatchRecipe();
    if (!r) return FB_FFT_ERR_ALLOC;
    const long long tw_elems = std::max(2LL, twb.total);
    if (cudaMalloc(&r->tw, (size_t)tw_elems * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        return FB_FFT_ERR_ALLOC;
    }
    for (const TwiddleJob& j : twb.jobs) {
        const cudaError_t e = launch_twiddles(r->tw, j, stream);
        if (e != cudaSuccess) {
            recipe_free(r);
            return cuda_fail(e, "recipe twiddles");
        }
    }
    r->table_bytes = tw_elems * (long long)sizeof(float2);
    r->scratch_bytes = scratch * (long long)sizeof(float2);
    r->scale = (float)(1.0 / (double)N);
    for (const PassPlan& q : passes) {
        BatchJob j;
        j.d = q.d;
        j.d.tw = r->tw;
        if (j.d.ptw) {
            j.d.ptw_lo = r->tw + reinterpret_cast<long long>(q.d.ptw_lo);
            j.d.ptw_hi = r->tw + reinterpret_cast<long long>(q.d.ptw_hi);
        }
        j.d.in = nullptr;
        j.d.out = nullptr;
        j.d.apply_scale = q.last ? 1 : 0;
        j.d.scale = r->scale;
        j.phase = q.group;
        j.src = q.src == kBufIn ? 0 : (q.src == kBufOut ? 1 : 2);
        j.dst = q.dst == kBufOut ? 1 : 2;
        j.last = q.last;
        const int padded = (int)(((long long)q.d.LS * (1LL << q.d.logT) + 15) & ~15LL);
        j.land = std::max(q.d.land_stride, padded);  // also serves as a work buffer
        j.work = padded;
        r->jobs.push_back(j);
        r->phases = std::max(r->phases, q.group + 1);
        r->tiles += q.d.ntiles;
    }
    *out = r;
    return FB_FFT_OK;
}

void recipe_free(BatchRecipe* r)
{
    if (!r) return;
    if (r->tw) cudaFree(r->tw);
    delete r;
}

// Resident CTAs of k_fft_uneven (or its inline form) on the current device
// for one shared-memory size, asked once per (device, size, form).
int uneven_resident(bool forward, size_t smem, bool inl, long long* cap)
{
    static std::mutex mu;
    static std::map<std::tuple<int, size_t, bool>, long long> fit;
    int dev = 0;
    FB_CK(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = fit.find({dev, smem, inl});
        if (it != fit.end()) {
            *cap = it->second;
            return FB_FFT_OK;
        }
    }
    int occ = 0, sms = 0;
    FB_CK(inl ? uneven_occupancy_inline(forward, smem, &occ) : uneven_occupancy(forward, smem, &occ));
    FB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (occ < 1) return cuda_fail(cudaErrorInvalidConfiguration, "batch launch occupancy");
    *cap = (long long)occ * sms;
    std::lock_guard<std::mutex> lock(mu);
    fit[{dev, smem, inl}] = *cap;
    return FB_FFT_OK;
}

int batch_launch(bool forward, const PassDesc* jobs, const int* tile_start, int njobs, long long tiles,
                 int land_max, int work_max, cudaStream_t stream)
{
    if (njobs <= 0 || tiles <= 0) return FB_FFT_OK;
    if (tiles >= (1LL << 31)) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    const size_t smem = uneven_smem_bytes(land_max, work_max);
    long long cap = 0;
    int rc = uneven_resident(forward, smem, false, &cap);
    if (rc != FB_FFT_OK) return rc;
    UnevenArgs a;
    a.jobs = jobs;
    a.tile_start = tile_start;
    a.in = nullptr;
    a.out = nullptr;
    a.scratch = nullptr;
    a.njobs = njobs;
    a.land_max = land_max;
    a.work_max = work_max;
    a.scale_on = 1;  // each job's apply_scale says whether it scales
    const cudaError_t e = uneven_launch(forward, a, std::min(tiles, cap), smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "k_fft_uneven (server batch)");
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return FB_FFT_OK;
}

int batch_launch_inline(bool forward, const PassDesc* jobs, const int* tile_start, int njobs, long long tiles,
                        int land_max, int work_max, cudaStream_t stream)
{
    if (njobs <= 0 || tiles <= 0) return FB_FFT_OK;
    if (njobs > kUnevenInlineJobs) return FB_FFT_ERR_INVALID_ARG;
    if (tiles >= (1LL << 31)) return FB_FFT_ERR_UNSUPPORTED_SIZE;
    const size_t smem = uneven_smem_bytes(land_max, work_max);
    long long cap = 0;
    int rc = uneven_resident(forward, smem, true, &cap);
    if (rc != FB_FFT_OK) return rc;
    UnevenInlineArgs p;
    std::memset(&p, 0, sizeof(p));
    p.a.njobs = njobs;
    p.a.land_max = land_max;
    p.a.work_max = work_max;
    p.a.scale_on = 1;
    std::memcpy(p.jobs, jobs, (size_t)njobs * sizeof(PassDesc));
    std::memcpy(p.tile_start, tile_start, (size_t)(njobs + 1) * sizeof(int));
    const cudaError_t e = uneven_launch_inline(forward, p, std::min(tiles, cap), smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "k_fft_uneven_inline (server batch)");
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return FB_FFT_OK;
}

int fail(cudaError_t e, const char* what) { return cuda_fail(e, what); }

}  // namespace host
}  // namespace fbfft

extern "C" {

const char* fb_fft_last_error(void) { return g_last_error; }

const char* fb_fft_status_string(int status)
{
    switch (status) {
    case FB_FFT_OK: return "ok";
    case FB_FFT_ERR_INVALID_ARG: return "invalid argument";
    case FB_FFT_ERR_UNSUPPORTED_SIZE: return "unsupported size (dims must be 5-smooth and within limits)";
    case FB_FFT_ERR_ALLOC: return "allocation failed";
    case FB_FFT_ERR_CUDA: return "CUDA error";
    case FB_FFT_ERR_TIMEOUT: return "device wait timed out";
    case FB_FFT_ERR_BAD_PLAN: return "bad plan handle";
    case FB_FFT_ERR_NO_DEVICE: return "no CUDA device";
    case FB_FFT_ERR_CANCELLED: return "request cancelled";
    case FB_FFT_ERR_OVER_BUDGET: return "request exceeds the server's device-memory budget";
    default: return "unknown status";
    }
}

int fb_fft_factorize(long long n, int* radices, int capacity, int* count)
{
    if (!count || (capacity > 0 && !radices) || capacity < 0) return FB_FFT_ERR_INVALID_ARG;
    int c = factorize(n, radices, capacity);
    if (c < 0) return c;
    *count = c;
    return c <= capacity ? FB_FFT_OK : FB_FFT_ERR_INVALID_ARG;
}

int fb_fft_split(long long n, long long* n1, long long* n2)
{
    if (!n1 || !n2) return FB_FFT_ERR_INVALID_ARG;
    return split_fourstep(n, n1, n2);
}

int fb_fft_plan_query(int rank, const long long* dims, long long batch, unsigned flags, fb_fft_info* info)
{
    if (!info) return FB_FFT_ERR_INVALID_ARG;
    long long N = 1;
    int rc = validate(rank, dims, batch, flags, &N);
    if (rc != FB_FFT_OK) return rc;
    fb_fft_plan_s p;
    p.rank = rank;
    for (int d = 0; d < rank; ++d) p.dims[d] = dims[d];
    p.batch = batch;
    p.flags = flags;
    p.N = N;
    TwiddleBuilder twb;
    rc = schedule_plan(&p, twb);
    p.magic = kDead;
    if (rc != FB_FFT_OK) return rc;
    std::memset(info, 0, sizeof(*info));
    info->passes = (int)p.passes.size();
    info->tc_passes = tc_pass_count(p.passes);
    info->smem_len_max = p.smem_len_max;
    info->scratch_bytes = (long long)p.scratch_bytes;
    info->twiddle_bytes = p.tw_elems * (long long)sizeof(float2);
    info->elements = N;
    info->batch = batch;
    return FB_FFT_OK;
}

int fb_fft_plan(fb_fft_plan_t* plan, int rank, const long long* dims, long long batch, unsigned flags,
                void* stream)
{
    if (!plan) return FB_FFT_ERR_INVALID_ARG;
    return plan_new(plan, rank, dims, batch, flags, (cudaStream_t)stream, false);
}

long long fb_fft_many_layout(int count, const long long* lengths, long long* offsets)
{
    if (count < 0 || (count > 0 && !lengths)) return -1;
    for (int i = 0; i < count; ++i)
        if (lengths[i] < 1) return -1;
    return many_layout(count, lengths, offsets);
}

int fb_fft_plan_many_ex(fb_fft_plan_t* plan, int count, const long long* lengths, unsigned flags, void* stream,
                        const fb_fft_many_opts* opts)
{
    if (!plan) return FB_FFT_ERR_INVALID_ARG;
    *plan = nullptr;
    if (count < 0 || (count > 0 && !lengths) || (flags & ~FB_FFT_SCALE_INV_N)) return FB_FFT_ERR_INVALID_ARG;
    if (opts && (opts->streams < 0 || opts->streams > 32 || opts->chunk_bytes < 0 || opts->max_lines < 0))
        return FB_FFT_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        if (lengths[i] < 1) return FB_FFT_ERR_INVALID_ARG;
        long long n1, n2;
        const int rc = split_fourstep(lengths[i], &n1, &n2);
        if (rc != FB_FFT_OK) return rc;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return FB_FFT_ERR_NO_DEVICE;
    }
    fb_fft_plan_s* p = new (std::nothrow) fb_fft_plan_s();
    if (!p) return FB_FFT_ERR_ALLOC;
    cudaGetDevice(&p->device);
    p->many = true;
    p->rank = 1;
    p->batch = count;
    p->flags = flags;
    p->stream = (cudaStream_t)stream;
    p->lengths.assign(lengths, lengths + count);
    p->offsets.resize(count);
    p->total = many_layout(count, lengths, p->offsets.data());
    p->N = 0;
    p->nslots = (opts && opts->streams > 0) ? opts->streams : many_streams();
    if (opts) {
        if (opts->use_graph == 0 || opts->use_graph == 1) p->use_graph = opts->use_graph == 1;
        p->chunk_bytes = opts->chunk_bytes;
        p->odd_first = opts->odd_radices_first != 0;
        p->max_lines = opts->max_lines;
        p->merge_mixed = opts->per_length == 0;
    }
    p->uneven = use_uneven_engine(count, lengths, opts);
    p->uneven_one = p->uneven && !(opts && opts->engine == 2);
    int rc = build_plan(p);
    if (rc != FB_FFT_OK) {
        free_plan(p);
        return rc;
    }
    *plan = p;
    return FB_FFT_OK;
}

int fb_fft_plan_many(fb_fft_plan_t* plan, int count, const long long* lengths, unsigned flags, void* stream)
{
    return fb_fft_plan_many_ex(plan, count, lengths, flags, stream, nullptr);
}

int fb_fft_autotune_many(int count, const long long* lengths, unsigned flags, const void* in, void* out,
                         int direction, void* stream, int reps, fb_fft_many_opts* best, float* best_ms)
{
    if (!best || !best_ms || reps < 1 || !in || !out) return FB_FFT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    FB_CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaErrorUnknown, "cudaEventCreate");
    }
    auto measure = [&](const fb_fft_many_opts& o, float* ms) -> int {
        fb_fft_plan_t pl = nullptr;
        int rc = fb_fft_plan_many_ex(&pl, count, lengths, flags, stream, &o);
        if (rc != FB_FFT_OK) return rc;
        for (int w = 0; w < 2 && rc == FB_FFT_OK; ++w) rc = fb_fft_exec(pl, in, out, direction);
        if (rc == FB_FFT_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = FB_FFT_ERR_CUDA;
        for (int r = 0; r < reps && rc == FB_FFT_OK; ++r) rc = fb_fft_exec(pl, in, out, direction);
        if (rc == FB_FFT_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            rc = FB_FFT_ERR_CUDA;
        float t = 0.f;
        if (rc == FB_FFT_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = FB_FFT_ERR_CUDA;
        if (rc == FB_FFT_OK) rc = fb_fft_check(pl);
        fb_fft_destroy(pl);
        *ms = t / reps;
        return rc;
    };
    // engine 0 (one kernel, one launch): its knob is the chunk size; then the
    // same kernel in one launch per phase (engine 2) at the best chunk size
    const long long chunks[] = {8LL << 20, 16LL << 20, 64LL << 20, 128LL << 20, 512LL << 20};
    fb_fft_many_opts best0{4, 1, 512LL << 20, 0, 0, 0, 0};  // engine 1's knobs at their defaults
    float best0_ms = 0.f;
    int rc = FB_FFT_OK;
    bool have0 = false;
    if (use_uneven_engine(count, lengths, nullptr)) {
        rc = measure(best0, &best0_ms);
        have0 = rc == FB_FFT_OK;
        for (long long v : chunks) {
            if (rc != FB_FFT_OK || v == best0.chunk_bytes) continue;
            fb_fft_many_opts o = best0;
            o.chunk_bytes = v;
            float ms;
            rc = measure(o, &ms);
            if (rc == FB_FFT_OK && ms < best0_ms) best0 = o, best0_ms = ms;
        }
        if (rc == FB_FFT_OK) {
            fb_fft_many_opts o = best0;
            o.engine = 2;
            float ms;
            rc = measure(o, &ms);
            if (rc == FB_FFT_OK && ms < best0_ms) best0 = o, best0_ms = ms;
        }
    }
    // engine 1 (per-kernel launches on side streams): coordinate descent, one knob at a time
    fb_fft_many_opts cur{4, 1, 32LL << 20, 0, 0, 0, 1};
    float cur_ms = 0.f;
    if (rc == FB_FFT_OK) rc = measure(cur, &cur_ms);
    const int streams[] = {1, 2, 8, 16, 32};
    const int lines[] = {4, 16, 64};
    for (int v : streams) {
        if (rc != FB_FFT_OK) break;
        fb_fft_many_opts o = cur;
        o.streams = v;
        float ms;
        rc = measure(o, &ms);
        if (rc == FB_FFT_OK && ms < cur_ms) cur = o, cur_ms = ms;
    }
    for (long long v : chunks) {
        if (rc != FB_FFT_OK) break;
        fb_fft_many_opts o = cur;
        o.chunk_bytes = v;
        float ms;
        rc = measure(o, &ms);
        if (rc == FB_FFT_OK && ms < cur_ms) cur = o, cur_ms = ms;
    }
    if (rc == FB_FFT_OK) {
        fb_fft_many_opts o = cur;
        o.odd_radices_first = 1;
        float ms;
        rc = measure(o, &ms);
        if (rc == FB_FFT_OK && ms < cur_ms) cur = o, cur_ms = ms;
    }
    for (int v : lines) {
        if (rc != FB_FFT_OK) break;
        fb_fft_many_opts o = cur;
        o.max_lines = v;
        float ms;
        rc = measure(o, &ms);
        if (rc == FB_FFT_OK && ms < cur_ms) cur = o, cur_ms = ms;
    }
    if (rc == FB_FFT_OK) {
        fb_fft_many_opts o = cur;
        o.per_length = 1;
        float ms;
        rc = measure(o, &ms);
        if (rc == FB_FFT_OK && ms < cur_ms) cur = o, cur_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FB_FFT_OK) return rc;
    if (have0 && best0_ms <= cur_ms) cur = best0, cur_ms = best0_ms;
    *best = cur;
    *best_ms = cur_ms;
    return FB_FFT_OK;
}

int fb_fft_plan_many_query(int count, const long long* lengths, unsigned flags, fb_fft_info* info)
{
    if (!info || count < 0 || (count > 0 && !lengths) || (flags & ~FB_FFT_SCALE_INV_N)) return FB_FFT_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        if (lengths[i] < 1) return FB_FFT_ERR_INVALID_ARG;
        long long n1, n2;
        const int rc = split_fourstep(lengths[i], &n1, &n2);
        if (rc != FB_FFT_OK) return rc;
    }
    fb_fft_plan_s p;
    p.many = true;
    p.rank = 1;
    p.batch = count;
    p.flags = flags;
    p.lengths.assign(lengths, lengths + count);
    p.offsets.resize(count);
    p.total = many_layout(count, lengths, p.offsets.data());
    p.nslots = many_streams();
    p.uneven = use_uneven_engine(count, lengths, nullptr);
    p.uneven_one = p.uneven;
    TwiddleBuilder twb;
    const int rc = schedule_plan(&p, twb);
    p.magic = kDead;
    if (rc != FB_FFT_OK) return rc;
    std::memset(info, 0, sizeof(*info));
    info->passes = (int)launches_per_exec(&p);
    info->tc_passes = tc_pass_count(p.passes);
    info->smem_len_max = p.smem_len_max;
    info->scratch_bytes = (long long)p.scratch_bytes;
    info->twiddle_bytes = p.tw_elems * (long long)sizeof(float2);
    info->elements = p.total;
    info->batch = count;
    return FB_FFT_OK;
}

int fb_fft_set_graph(fb_fft_plan_t plan, int enable)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    plan->use_graph = enable != 0;
    return FB_FFT_OK;
}

int fb_fft_exec(fb_fft_plan_t plan, const void* in, void* out, int direction)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    if (direction != FB_FFT_FORWARD && direction != FB_FFT_INVERSE) return FB_FFT_ERR_INVALID_ARG;
    if (plan->batch == 0) return FB_FFT_OK;
    if (!in || !out) return FB_FFT_ERR_INVALID_ARG;
    if (((uintptr_t)in | (uintptr_t)out) & 7) return FB_FFT_ERR_INVALID_ARG;
    const uintptr_t bytes = (uintptr_t)plan_elems(plan) * sizeof(float2);
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a != b && a < b + bytes && b < a + bytes) return FB_FFT_ERR_INVALID_ARG;
    return exec_device(plan, (const float2*)in, (float2*)out, direction);
}

int fb_fft_exec_host(fb_fft_plan_t plan, const void* host_in, void* host_out, int direction)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    if (direction != FB_FFT_FORWARD && direction != FB_FFT_INVERSE) return FB_FFT_ERR_INVALID_ARG;
    if (plan->batch == 0) return FB_FFT_OK;
    if (!host_in || !host_out) return FB_FFT_ERR_INVALID_ARG;
    const size_t bytes = (size_t)plan_elems(plan) * sizeof(float2);
    if (!plan->staging) {
        if (cudaMalloc(&plan->staging, bytes) != cudaSuccess) {
            cudaGetLastError();
            plan->staging = nullptr;
            return FB_FFT_ERR_ALLOC;
        }
        plan->staging_bytes = bytes;
    }
    const long long cb = host_chunk_batch(plan, host_in, host_out);
    if (cb > 0) return exec_host_pipelined(plan, (const float2*)host_in, (float2*)host_out, direction, cb);
    FB_CK(cudaMemcpyAsync(plan->staging, host_in, bytes, cudaMemcpyHostToDevice, plan->stream));
    int rc = exec_device(plan, plan->staging, plan->staging, direction);
    if (rc != FB_FFT_OK) return rc;
    FB_CK(cudaMemcpyAsync(host_out, plan->staging, bytes, cudaMemcpyDeviceToHost, plan->stream));
    return fb_fft_check(plan);
}

int fb_fft_check(fb_fft_plan_t plan)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    FB_CK(cudaStreamSynchronize(plan->stream));
    int e[4] = {0, 0, 0, 0};
    FB_CK(cudaMemcpy(e, plan->err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e[0]) {
        if (e[0] == 2)
            snprintf(g_last_error, sizeof(g_last_error), "self-check: copy kind %d at address ...%08x, %d bytes", e[1],
                     (unsigned)e[2], e[3]);
        cudaMemset(plan->err, 0, 16 * sizeof(int));
        return FB_FFT_ERR_TIMEOUT;
    }
    return FB_FFT_OK;
}

int fb_fft_debug_inject_timeout(fb_fft_plan_t plan, int enable)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    plan->debug_timeout = enable != 0;
    return FB_FFT_OK;
}

int fb_fft_offload_decide(fb_fft_plan_t plan, fb_fft_cpu_block cpu, void* ctx, const void* host_in, void* host_out,
                          int direction, int reps, int* use_gpu, double* cpu_ms, double* gpu_ms)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    if (!cpu || !host_in || !host_out || reps < 1 || !use_gpu || !cpu_ms || !gpu_ms) return FB_FFT_ERR_INVALID_ARG;
    if (direction != FB_FFT_FORWARD && direction != FB_FFT_INVERSE) return FB_FFT_ERR_INVALID_ARG;
    using clk = std::chrono::steady_clock;
    cpu(ctx, host_in, host_out, direction);  // untimed first call of each side
    int rc = fb_fft_exec_host(plan, host_in, host_out, direction);
    if (rc != FB_FFT_OK) return rc;
    auto t0 = clk::now();
    for (int r = 0; r < reps; ++r) cpu(ctx, host_in, host_out, direction);
    auto t1 = clk::now();
    for (int r = 0; r < reps && rc == FB_FFT_OK; ++r) rc = fb_fft_exec_host(plan, host_in, host_out, direction);
    auto t2 = clk::now();
    if (rc != FB_FFT_OK) return rc;
    *cpu_ms = std::chrono::duration<double, std::milli>(t1 - t0).count() / reps;
    *gpu_ms = std::chrono::duration<double, std::milli>(t2 - t1).count() / reps;
    *use_gpu = *gpu_ms < *cpu_ms ? 1 : 0;
    return FB_FFT_OK;
}

int fb_fft_set_stream(fb_fft_plan_t plan, void* stream)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    plan->stream = (cudaStream_t)stream;
    return FB_FFT_OK;
}

int fb_fft_destroy(fb_fft_plan_t plan)
{
    if (!plan) return FB_FFT_OK;
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    cudaStreamSynchronize(plan->stream);
    free_plan(plan);
    return FB_FFT_OK;
}

int fb_fft_plan_info(fb_fft_plan_t plan, fb_fft_info* info)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    if (!info) return FB_FFT_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->passes = (int)launches_per_exec(plan);
    info->tc_passes = tc_pass_count(plan->passes);
    info->smem_len_max = plan->smem_len_max;
    info->scratch_bytes = (long long)plan->scratch_bytes;
    info->twiddle_bytes = plan->tw_elems * (long long)sizeof(float2);
    info->elements = plan->many ? plan->total : plan->N;
    info->batch = plan->batch;
    return FB_FFT_OK;
}

int fb_fft_profile(fb_fft_plan_t plan, int enable)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    plan->profiling = enable != 0;
    plan->ev_used = 0;
    return FB_FFT_OK;
}

int fb_fft_profile_read(fb_fft_plan_t plan, double* ms_total, long long* launches, int capacity, int* npasses)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    if (!npasses || capacity < 0 || (capacity > 0 && (!ms_total || !launches))) return FB_FFT_ERR_INVALID_ARG;
    const int ng = (int)plan->group_names.size();
    *npasses = ng;
    for (int g = 0; g < capacity; ++g) ms_total[g] = 0.0, launches[g] = 0;
    if (plan->ev_used) {
        FB_CK(cudaEventSynchronize(plan->ev[plan->ev_used - 1]));
        for (size_t i = 0; i + 1 < plan->ev_used; i += 2) {
            float ms = 0.f;
            FB_CK(cudaEventElapsedTime(&ms, plan->ev[i], plan->ev[i + 1]));
            const int g = plan->ev_group[i / 2];
            if (g < capacity) ms_total[g] += ms, launches[g] += 1;
        }
    }
    plan->ev_used = 0;
    return FB_FFT_OK;
}

int fb_fft_pass_launch(fb_fft_plan_t plan, int pass, long long* grid, int* block, long long* smem_bytes)
{
    if (!plan_ok(plan)) return FB_FFT_ERR_BAD_PLAN;
    if (pass < 0 || pass >= (int)plan->passes.size() || !grid || !block || !smem_bytes) return FB_FFT_ERR_INVALID_ARG;
    const PassPlan& q = plan->passes[pass];
    *grid = q.grid;
    *block = pass_kernel(q, true).threads;
    *smem_bytes = (long long)q.smem;
    return FB_FFT_OK;
}

const char* fb_fft_pass_name(fb_fft_plan_t plan, int pass)
{
    if (!plan_ok(plan) || pass < 0 || pass >= (int)plan->group_names.size()) return nullptr;
    return plan->group_names[pass];
}

long long fb_fft_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int fb_fft_twiddles(long long d, long long count, float* host_out)
{
    if (d < 1 || count < 0 || (count > 0 && !host_out)) return FB_FFT_ERR_INVALID_ARG;
    if (count == 0) return FB_FFT_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return FB_FFT_ERR_NO_DEVICE;
    }
    float2* buf = nullptr;
    if (cudaMalloc(&buf, (size_t)count * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        return FB_FFT_ERR_ALLOC;
    }
    TwiddleJob j{0, count, d, 1, 0, 0, 0};
    int rc = FB_FFT_OK;
    cudaError_t e = launch_twiddles(buf, j, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(host_out, buf, (size_t)count * sizeof(float2), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "fb_fft_twiddles");
    cudaFree(buf);
    return rc;
}

}  // extern "C"
