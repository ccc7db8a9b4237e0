// fft_plane.cuh -- the plane pass: the 2-D DFT over the two trailing axes of
// a row-major array (Sec. 5.1(a)'s multi-dimensional transform as separable
// 1-D DFTs, two of its axis passes fused into one trip through HBM).
//
// A plane holds L1 rows of L2 contiguous values (L1, L2 in {128, 256}: 128
// to 512 KB), more than one CTA's shared memory.  A cluster of CS CTAs
// shares it through distributed shared memory:
//   1. CTA q loads rows [q*R1, (q+1)*R1) and runs their L2-point DFTs;
//   2. cluster barrier; CTA q owns columns [q*W, (q+1)*W) and reads the first
//      column stage's 16 inputs of each butterfly from the CTAs that hold
//      those rows (ld.shared::cluster);
//   3. cluster barrier (every buffer has been read); the butterflies'
//      outputs land in the CTA's own buffer as an L1 x W column block, the
//      second column stage runs there, and one TMA tensor store writes the
//      block to its W columns of the plane.
// Both 1-D transforms are two Stockham stages, radix 16 and then L/16
// (the same schedule and twiddle tables as the line passes).  Every compute
// thread holds 16 values per stage; TH compute threads (512: one CTA per SM;
// 256: two, from different clusters) hold R1 * L2 = 16 TH values, which fixes
// CS = L1 * L2 / (16 TH).
//
// Persistent clusters walk the planes (cluster id, + number of clusters).
// One producer warp per CTA keeps NBUF plane slices in flight: bulk row
// loads into buffer i % NBUF (mbarrier full), and once the compute warps
// have finished a plane (mbarrier done) the tensor store and the reload of
// that buffer.  Every CTA of a cluster runs the same number of iterations and
// every thread of it takes both cluster barriers of every iteration, bounded
// waits included (a wait that gives up records the error and carries on), so
// no CTA can leave its cluster waiting.
#pragma once

#include "fft_p2.cuh"  // compute_sync, mbar_arrive

namespace fbfft {

__host__ __device__ constexpr int plane_row_stride(int lg2)
{
    // >= L2 + L2/16 (the padded index spad of the first stage's outputs);
    // with G2 = L2/16 < 16 threads per row a half-warp covers 16/G2 rows,
    // which a stride of G2 (mod 16) values puts on disjoint banks
    const int l2 = 1 << lg2, g2 = l2 / 16;
    int rs = l2 + l2 / 16;
    if (g2 < 16)
        while (rs % 16 != g2) ++rs;
    return rs;
}

template <int LG1, int LG2, int TH = 512>
struct PlaneCfg {
    static constexpr int L1 = 1 << LG1;  // rows: length of the column DFTs
    static constexpr int L2 = 1 << LG2;  // row length (contiguous)
    static constexpr int THREADS = TH;   // compute threads: 512 (one CTA per SM) or 256 (two)
    static constexpr int E = 16;         // values per thread per stage
    static constexpr int CS = L1 * L2 / (THREADS * E);  // CTAs per cluster
    static constexpr int R1 = L1 / CS;   // rows per CTA
    static constexpr int W = L2 / CS;    // columns per CTA
    static constexpr int G2 = L2 / 16;   // radix of the rows' second stage (butterflies per row in the first)
    static constexpr int G1 = L1 / 16;   // the same for the columns
    static constexpr int RS = plane_row_stride(LG2);
    static constexpr int BUF = R1 * RS;  // elements of one plane-slice buffer
    static constexpr int NBUF = 3;
    static constexpr int TW_ROW = 16 * (G2 - 1);  // row stage-1 table: w_L2^{r k}, entry (r-1)*16 + k
    static constexpr int TW_COL = 16 * (G1 - 1);  // column stage-1 table: w_L1^{r k}
    static constexpr int ROWS_PER_OWNER = 16 / CS;  // first-stage inputs of a column butterfly per CTA
    static constexpr long long SMEM = 128 + 128 + 8LL * (NBUF * BUF + TW_ROW + TW_COL);

    static_assert(CS == 1 || CS == 2 || CS == 4 || CS == 8, "cluster of 1, 2, 4 or 8 CTAs");
    static_assert(G1 >= 2 && G1 <= 16 && G2 >= 2 && G2 <= 16, "two-stage schedules (radix 16, then L/16)");
    static_assert(R1 * L2 == THREADS * E && L1 * W == THREADS * E, "one stage of 16 values per thread");
    static_assert(W % 16 == 0, "half-warps cover 16 consecutive columns");
    static_assert(R1 % G1 == 0, "rows of a column butterfly split evenly over the CTAs");
    static_assert(L1 * W <= BUF, "the column block fits the row buffer");
    static_assert((BUF * 8) % 128 == 0 && RS % 2 == 0, "buffers and rows 128- and 16-byte aligned");
    static_assert(SMEM <= 227 * 1024, "shared memory");

    // Row phase: thread t owns row row_of(t) and first-stage butterfly rj_of(t).
    __host__ __device__ static constexpr int row_of(int t) { return t / G2; }
    __host__ __device__ static constexpr int rj_of(int t) { return t % G2; }
    // First row stage (radix 16, Ns = 1): input r of butterfly j sits at
    // n = j + G2 r of the dense row; output r goes to index 16 j + r, stored
    // padded (spad) in the same row.
    __host__ __device__ static constexpr int row_s0_in(int j, int r) { return j + G2 * r; }
    __host__ __device__ static constexpr int row_s0_out(int j, int r) { return (16 * j + r) + ((16 * j + r) >> 4); }
    // Second row stage (radix G2, Ns = 16): butterfly j < 16 reads and writes
    // index j + 16 r (padded); the thread's butterflies are rj + G2 u.
    __host__ __device__ static constexpr int row_s1(int j, int r) { return (j + 16 * r) + ((j + 16 * r) >> 4); }
    // Column phase: thread t owns column cl_of(t) of the CTA's W and butterfly cj_of(t).
    __host__ __device__ static constexpr int cl_of(int t) { return t % W; }
    __host__ __device__ static constexpr int cj_of(int t) { return t / W; }
    // First column stage (radix 16, Ns = 1): input r of butterfly j is row
    // j + G1 r, held by CTA owner(r) as its local row lrow(j, r).
    __host__ __device__ static constexpr int owner(int r) { return r / ROWS_PER_OWNER; }
    __host__ __device__ static constexpr int lrow(int j, int r) { return j + G1 * (r % ROWS_PER_OWNER); }
    // Slot of column c (0 <= c < L2) in a row-phase row.
    __host__ __device__ static constexpr int col_slot(int c) { return c + (c >> 4); }
    // Column block: value (row m, column cl) at m * W + cl; first-stage output
    // r of butterfly j is row 16 j + r, the second stage (radix G1, Ns = 16)
    // reads and writes rows j + 16 r.
    __host__ __device__ static constexpr int blk(int m, int cl) { return m * W + cl; }
};

__device__ __forceinline__ unsigned cluster_ctarank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_id_x()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_count_x()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// All threads of all CTAs of the cluster; release/acquire orders every
// shared-memory access before it against every access after it.
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The same barrier without ordering this thread's earlier accesses: for a
// thread whose earlier reads have all returned (their values are consumed)
// and whose writes nobody reads across it.
__device__ __forceinline__ void cluster_barrier_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned cluster_map(unsigned saddr, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_cluster(unsigned addr)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}

// Producer warp: bulk-load this CTA's R1 rows of `plane` into dst (row stride RS).
template <class P>
__device__ __forceinline__ void plane_issue_load(const PassDesc& d, long long plane, unsigned q, float2* dst,
                                                 unsigned long long* bar, int lane)
{
    const float2* src = d.in + plane * d.in_so + (long long)q * P::R1 * d.in_sn;
    if (lane == 0) mbar_arrive_expect_tx(bar, (unsigned)(P::R1 * P::L2 * 8) + d.debug_extra_tx);
    __syncwarp();
    for (int r = lane; r < P::R1; r += 32)
        bulk_load_1d(dst + r * P::RS, src + (long long)r * d.in_sn, (unsigned)(P::L2 * 8), bar, d.err);
}

// Row DFTs of the CTA's R1 rows, in place in `buf` (dense rows in, padded rows out).
template <class P, bool FWD>
__device__ __forceinline__ void plane_rows(float2* buf, const float2* twr)
{
    constexpr int G2 = P::G2;
    const int t = threadIdx.x;
    const int j0 = P::rj_of(t);
    float2* rp = buf + P::row_of(t) * P::RS;
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = rp[P::row_s0_in(j0, r)];
    compute_sync<P::THREADS>();  // every dense read is done before the padded writes
    dft<16, FWD>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) rp[P::row_s0_out(j0, r)] = v[r];
    compute_sync<P::THREADS>();
#pragma unroll
    for (int u = 0; u < 16 / G2; ++u) {
        const int j = j0 + G2 * u;
        float2 w[G2];
#pragma unroll
        for (int r = 0; r < G2; ++r) w[r] = rp[P::row_s1(j, r)];
#pragma unroll
        for (int r = 1; r < G2; ++r) w[r] = twmul<FWD>(w[r], twr[(r - 1) * 16 + j]);
        dft<G2, FWD>(w);
#pragma unroll
        for (int r = 0; r < G2; ++r) rp[P::row_s1(j, r)] = w[r];
    }
}

// The plane pass.  d.in / d.out: plane p's row n starts at p * so + n * sn
// (in_so/in_sn, out_so/out_sk); d.ntiles planes; d.twoff[0] / [1]: the row /
// column stage-1 twiddle tables; tm_out: view {L2, L1, planes}, box {W, L1, 1}.
template <int LG1, int LG2, int TH, bool FWD>
__global__ void __launch_bounds__(TH + 32, TH <= 256 ? 2 : 1) k_fft_plane(const __grid_constant__ LineArgs a)
{
    using P = PlaneCfg<LG1, LG2, TH>;
    constexpr int NBUF = P::NBUF;
    const PassDesc& d = a.d;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(smem_raw);  // [NBUF]
    unsigned long long* done = full + NBUF;                                       // [NBUF]
    float2* buf0 = reinterpret_cast<float2*>(smem_raw + 128);
    float2* twr = buf0 + NBUF * P::BUF;
    float2* twc = twr + P::TW_ROW;
    const bool async = d.async_io != 0;
    const unsigned q = cluster_ctarank();
    const long long cid = cluster_id_x(), ncl = cluster_count_x();
    const long long nplanes = d.ntiles;
    const int n = cid < nplanes ? (int)((nplanes - 1 - cid) / ncl + 1) : 0;  // planes of this cluster
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&done[b], P::THREADS);
        }
        fence_mbar_init();
    }
    __syncthreads();
    pdl_start();

    if (warp == P::THREADS / 32) {
        // ---- producer warp ----
        bool ok = true;
        if (async)
            for (int i = 0; i < NBUF && i < n; ++i)
                plane_issue_load<P>(d, cid + i * ncl, q, buf0 + i * P::BUF, &full[i], lane);
        for (int i = 0; i < n; ++i) {
            cluster_barrier();  // rows of plane i transformed in every CTA
            cluster_barrier();  // every CTA has read its column inputs of plane i
            if (!async) continue;
            const int b = i % NBUF;
            const bool got = mbar_wait_bounded(&done[b], (unsigned)(i / NBUF) & 1u);
            ok = ok && got;
            if (got && lane == 0) {
                tma_store_3d(&a.tm_out, (int)q * P::W, 0, (int)(cid + i * ncl), buf0 + b * P::BUF, d.err);
                bulk_commit();
            }
            if (i + NBUF < n) {
                if (lane == 0) bulk_wait_read_all();  // the store has read the buffer
                __syncwarp();
                plane_issue_load<P>(d, cid + (i + NBUF) * ncl, q, buf0 + b * P::BUF, &full[b], lane);
            }
        }
        if (!ok && lane == 0) atomicExch(d.err, 1);
        if (lane == 0) bulk_wait_all();
        return;
    }

    // ---- compute warps ----
    const int t = threadIdx.x;
    for (int e = t; e < P::TW_ROW; e += P::THREADS) twr[e] = __ldg(d.tw + d.twoff[0] + e);
    for (int e = t; e < P::TW_COL; e += P::THREADS) twc[e] = __ldg(d.tw + d.twoff[1] + e);
    compute_sync<P::THREADS>();
    const int cl = P::cl_of(t), cj = P::cj_of(t);
    const int cslot = P::col_slot((int)q * P::W + cl);
    unsigned rbase[P::CS];  // buffer 0 of every CTA of the cluster
#pragma unroll
    for (int o = 0; o < P::CS; ++o) rbase[o] = cluster_map(smem_u32(buf0), (unsigned)o);
    bool bad = false;
    for (int i = 0; i < n; ++i) {
        const long long plane = cid + i * ncl;
        const int b = async ? i % NBUF : 0;
        float2* buf = buf0 + b * P::BUF;
        if (async) {
            if (!mbar_wait_bounded(&full[b], (unsigned)(i / NBUF) & 1u)) bad = true;  // carry on: barriers stay matched
        } else {
            const float2* src = d.in + plane * d.in_so + (long long)q * P::R1 * d.in_sn;
            for (int e = t; e < P::R1 * P::L2; e += P::THREADS) {
                const int r = e >> LG2, c = e & (P::L2 - 1);
                buf[r * P::RS + c] = src[(long long)r * d.in_sn + c];
            }
            compute_sync<P::THREADS>();
        }
        plane_rows<P, FWD>(buf, twr);
        cluster_barrier();
        // first column stage: gather the 16 inputs from the CTAs that hold the rows
        float2 v[16];
        const unsigned boff = (unsigned)(b * P::BUF) * 8u;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int o = P::owner(r);
            const int s = P::lrow(cj, r) * P::RS + cslot;
            v[r] = (o == (int)q) ? buf[s] : ld_cluster(rbase[o] + boff + (unsigned)s * 8u);
        }
        dft<16, FWD>(v);  // consumes every value read: the reads have returned
        cluster_barrier_relaxed();
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[P::blk(16 * cj + r, cl)] = v[r];
        compute_sync<P::THREADS>();
        // second column stage, in place in the column block
#pragma unroll
        for (int u = 0; u < 16 / P::G1; ++u) {
            const int j = cj + P::G1 * u;
            float2 w[P::G1];
#pragma unroll
            for (int r = 0; r < P::G1; ++r) w[r] = buf[P::blk(j + 16 * r, cl)];
#pragma unroll
            for (int r = 1; r < P::G1; ++r) w[r] = twmul<FWD>(w[r], twc[(r - 1) * 16 + j]);
            dft<P::G1, FWD>(w);
#pragma unroll
            for (int r = 0; r < P::G1; ++r) buf[P::blk(j + 16 * r, cl)] = d.apply_scale ? d.scale * w[r] : w[r];
        }
        if (async) {
            fence_proxy_async();  // the column block -> visible to the TMA store
            mbar_arrive(&done[b]);
        } else {
            compute_sync<P::THREADS>();
            float2* dst = d.out + plane * d.out_so + (long long)q * P::W;
            for (int e = t; e < P::L1 * P::W; e += P::THREADS) {
                const int m = e / P::W, c = e % P::W;
                dst[(long long)m * d.out_sk + c] = buf[e];
            }
            compute_sync<P::THREADS>();  // the buffer is read before the next plane's load
        }
    }
    if (bad && t == 0) atomicExch(d.err, 1);
}

template <int LG1, int LG2, int TH, bool FWD>
LineKernel plane_entry()
{
    using P = PlaneCfg<LG1, LG2, TH>;
    LineKernel k = make_entry<P::THREADS>(k_fft_plane<LG1, LG2, TH, FWD>, FWD, LG2, -1);
    k.threads = P::THREADS + 32;
    k.producers = 32;
    k.kind = 3;
    k.lg1 = LG1;
    k.cluster = P::CS;
    return k;
}

}  // namespace fbfft
