// fb_serve.cu -- request server of the FFT function block: continuous
// batching of offload calls over a fixed set of stream slots, admission by a
// device-memory budget, resident plans (C ABI in include/fb_fft.h).
//
// Life of a request:
//   submit   resolve the resident plan of its shape (build on a miss), size
//            its device needs (four-step scratch + staging for host arrays),
//            reject it when that exceeds the whole arena, else queue it (FIFO).
//   admit    the FIFO head goes to the first free slot once the arena can
//            hold its needs: staging copy in, plan passes, staging copy out,
//            all on the slot's stream, then a completion event.
//   retire   a slot whose event has completed returns its arena block, reads
//            its bounded-wait error word and appends the request to the done
//            list; the slot is free for the next admission at once.
// Every submit / poll / drain runs retire-then-admit, so requests arriving
// while others are on the GPU start as soon as a slot and memory free up.
//
// Batching: shapes whose axes (or four-step factors) fit one job of the
// one-kernel engine (k_fft_uneven) have a resident recipe of job
// descriptors.  When a slot frees up, admission takes the whole FIFO prefix
// of such requests that fits the budget (up to max_batch), writes their jobs
// with the requests' own addresses into the slot's pinned job table, copies
// it to the device with one copy and runs it as one launch per phase and
// direction (at most six).  Host work per request is then filling two or
// three descriptors instead of encoding tensor maps and launching kernels;
// the batch grows by itself with the queue, so an idle server still starts
// each request at once.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "fb_fft.h"
#include "fb_host.h"
#include "fft_uneven.cuh"

using namespace fbfft;

namespace {

constexpr uint32_t kServerMagic = 0x5E2FFB01u;
constexpr long long kArenaAlign = 256;

#define SV_CK(call)                                                       \
    do {                                                                  \
        cudaError_t sv_e_ = (call);                                       \
        if (sv_e_ != cudaSuccess) return host::fail(sv_e_, #call);        \
    } while (0)

// First-fit allocator over one device region; blocks are 256-byte aligned and
// free neighbours coalesce, so the budget is the region and nothing else.
struct Arena {
    char* base = nullptr;
    long long cap = 0, used = 0, peak = 0;
    std::map<long long, long long> free_;  // offset -> size

    void reset(long long c)
    {
        cap = c;
        free_.clear();
        if (c > 0) free_[0] = c;
    }
    long long alloc(long long n)  // offset, or -1
    {
        n = (n + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const long long off = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[off + n] = rest;
            used += n;
            peak = std::max(peak, used);
            return off;
        }
        return -1;
    }
    void release(long long off, long long n)
    {
        n = (n + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct ShapeKey {
    int rank;
    long long d0, d1, d2, batch;
    unsigned flags;
    bool operator<(const ShapeKey& o) const
    {
        if (rank != o.rank) return rank < o.rank;
        if (d0 != o.d0) return d0 < o.d0;
        if (d1 != o.d1) return d1 < o.d1;
        if (d2 != o.d2) return d2 < o.d2;
        if (batch != o.batch) return batch < o.batch;
        return flags < o.flags;
    }
};

struct PlanEntry {
    fb_fft_plan_t plan = nullptr;
    host::BatchRecipe* recipe = nullptr;  // null: this shape runs per request
    unsigned flags = 0;
    long long scratch = 0, io = 0, table = 0;
    long long last_use = 0;
    int users = 0;  // queued + running requests holding it
};

// Jobs one slot's table holds (a batch of up to 1024 jobs: 341 four-step or
// 3-D requests, more of the others).
constexpr int kBatchJobs = 1024;
constexpr int kBatchGroups = 6;  // launches per batch: three phases x two directions
constexpr size_t kTableBytes =
    ((kBatchJobs * sizeof(PassDesc) + (kBatchJobs + kBatchGroups) * sizeof(int)) + 255) / 256 * 256;

struct Req {
    long long tag = 0;
    PlanEntry* pe = nullptr;
    int direction = FB_FFT_FORWARD;
    const void* in = nullptr;
    void* out = nullptr;
    bool host_io = false;
    bool batched = false;  // runs through its shape's recipe in a batch
    long long need = 0;    // arena bytes
    double t_submit = 0, t_admit = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr;  // device time the request's work begins
    cudaEvent_t done = nullptr;   // ... and ends (the completion the server polls)
    int* err_dev = nullptr;   // int[16] bounded-wait error word of this slot's launches
    int* err_host = nullptr;  // pinned copy, refreshed at the end of every request
    bool err_mapped = false;  // err_dev is err_host mapped into the device: no copy per request
    bool busy = false;
    std::vector<Req> reqs;        // the request on this slot, or the batch
    std::vector<long long> offs;  // their arena blocks (-1: none)
    long long seq = 0;            // admission order
    char* tab_host = nullptr;     // batch job table: written here (pinned) ...
    char* tab_dev = nullptr;      // ... and copied here for the launches
};

}  // namespace

struct fb_fft_server_s {
    uint32_t magic = kServerMagic;
    int device = 0;
    int max_plans = 1;
    std::chrono::steady_clock::time_point t0;
    cudaStream_t build = nullptr;  // plans are built here
    cudaEvent_t ref = nullptr;     // device-clock origin of the done records' device times
    Arena arena;
    std::vector<Slot> slots;
    std::map<ShapeKey, PlanEntry> plans;
    std::deque<Req> pending;
    std::deque<fb_fft_server_done> done;
    long long use_clock = 0, seq = 0;
    int max_batch = 64;  // requests per batch; <= 1: every request alone through its plan
    int busy_slots = 0;
    fb_fft_server_stats st{};
};

namespace {

bool server_ok(fb_fft_server_t s) { return s && s->magic == kServerMagic; }

double now_s(const fb_fft_server_s* s)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

void evict_idle(fb_fft_server_s* s)
{
    while ((int)s->plans.size() > s->max_plans) {
        auto victim = s->plans.end();
        for (auto it = s->plans.begin(); it != s->plans.end(); ++it)
            if (it->second.users == 0 && (victim == s->plans.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == s->plans.end()) return;  // every plan is in use
        s->st.plan_bytes -= victim->second.table;
        host::plan_free(victim->second.plan);
        host::recipe_free(victim->second.recipe);
        s->plans.erase(victim);
    }
}

int get_plan(fb_fft_server_s* s, int rank, const long long* dims, long long batch, unsigned flags, PlanEntry** out)
{
    if (rank < 1 || rank > 3 || !dims) return FB_FFT_ERR_INVALID_ARG;
    ShapeKey k{rank, dims[0], rank > 1 ? dims[1] : 1, rank > 2 ? dims[2] : 1, batch, flags};
    auto it = s->plans.find(k);
    if (it == s->plans.end()) {
        PlanEntry e;
        int rc = host::plan_create(&e.plan, rank, dims, batch, flags, s->build, true);
        if (rc != FB_FFT_OK) return rc;
        e.flags = flags;
        e.scratch = host::plan_scratch_bytes(e.plan);
        e.io = host::plan_io_bytes(e.plan);
        e.table = host::plan_table_bytes(e.plan);
        // the batch recipe; a shape it cannot take runs per request
        rc = host::recipe_create(&e.recipe, rank, dims, batch, flags, s->build);
        if (rc == FB_FFT_ERR_UNSUPPORTED_SIZE) {
            e.recipe = nullptr;
        } else if (rc != FB_FFT_OK) {
            host::plan_free(e.plan);
            return rc;
        } else if ((long long)e.recipe->jobs.size() > kBatchJobs) {
            host::recipe_free(e.recipe);
            e.recipe = nullptr;
        }
        if (e.recipe) e.table += e.recipe->table_bytes;
        // the twiddle tables are written on the build stream; requests run on
        // the slots' streams, so the tables must be complete before the first
        const cudaError_t se = cudaStreamSynchronize(s->build);
        if (se != cudaSuccess) {
            host::plan_free(e.plan);
            host::recipe_free(e.recipe);
            return host::fail(se, "plan build");
        }
        s->st.plan_builds++;
        s->st.plan_bytes += e.table;
        it = s->plans.emplace(k, e).first;
    }
    it->second.last_use = ++s->use_clock;
    *out = &it->second;
    return FB_FFT_OK;
}

long long up_align(long long n) { return (n + kArenaAlign - 1) / kArenaAlign * kArenaAlign; }

long long scratch_of(const PlanEntry* pe, bool batched)
{
    return batched ? pe->recipe->scratch_bytes : pe->scratch;
}

long long request_need(const PlanEntry* pe, bool host_io, bool batched)
{
    return up_align(scratch_of(pe, batched)) + (host_io ? up_align(pe->io) : 0);
}

// Report every request on the slot done with `status` and free the slot.
void finish(fb_fft_server_s* s, Slot& sl, int slot_index, int status)
{
    const double t = now_s(s);
    double dev0 = -1.0, dev1 = -1.0;
    float a = 0.f, b = 0.f;
    if (status == FB_FFT_OK && cudaEventElapsedTime(&a, s->ref, sl.start) == cudaSuccess &&
        cudaEventElapsedTime(&b, s->ref, sl.done) == cudaSuccess) {
        dev0 = a * 1e-3;
        dev1 = b * 1e-3;
    }
    cudaGetLastError();
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        const Req& r = sl.reqs[i];
        fb_fft_server_done d;
        d.tag = r.tag;
        d.status = status;
        d.slot = slot_index;
        d.t_submit = r.t_submit;
        d.t_admit = r.t_admit;
        d.t_done = t;
        d.t_dev_start = dev0;
        d.t_dev_end = dev1;
        s->done.push_back(d);
        if (sl.offs[i] >= 0) s->arena.release(sl.offs[i], r.need);
        r.pe->users--;
        s->st.completed++;
        s->st.in_flight--;
    }
    sl.reqs.clear();
    sl.offs.clear();
    sl.busy = false;
    s->busy_slots--;
}

// Retire every slot whose completion event has fired.
int retire(fb_fft_server_s* s)
{
    for (int i = 0; i < (int)s->slots.size(); ++i) {
        Slot& sl = s->slots[i];
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) {
            cudaGetLastError();
            continue;
        }
        int status = FB_FFT_OK;
        if (q != cudaSuccess) {
            status = host::fail(q, "request completion");
        } else if (*static_cast<volatile int*>(sl.err_host) != 0) {
            status = FB_FFT_ERR_TIMEOUT;
            std::memset(sl.err_host, 0, 16 * sizeof(int));
            if (!sl.err_mapped) {
                const cudaError_t e = cudaMemsetAsync(sl.err_dev, 0, 16 * sizeof(int), sl.stream);
                if (e != cudaSuccess) status = host::fail(e, "cudaMemsetAsync");
            }
        }
        finish(s, sl, i, status);
    }
    return FB_FFT_OK;
}

// Put request r on slot sl: copies and passes on the slot's stream, then its event.
int start(fb_fft_server_s* s, Slot& sl, const Req& r, long long off)
{
    (void)s;
    char* block = off >= 0 ? s->arena.base + off : nullptr;
    const long long scr_bytes = (r.pe->scratch + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    void* scratch = r.pe->scratch ? block : nullptr;
    const void* in = r.in;
    void* out = r.out;
    SV_CK(cudaEventRecord(sl.start, sl.stream));
    if (r.host_io) {
        void* stage = block + scr_bytes;
        SV_CK(cudaMemcpyAsync(stage, r.in, (size_t)r.pe->io, cudaMemcpyHostToDevice, sl.stream));
        in = stage;
        out = stage;
    }
    int rc = host::plan_exec_on(r.pe->plan, in, out, r.direction, sl.stream, scratch, sl.err_dev);
    if (rc != FB_FFT_OK) return rc;
    if (r.host_io) SV_CK(cudaMemcpyAsync(r.out, out, (size_t)r.pe->io, cudaMemcpyDeviceToHost, sl.stream));
    if (!sl.err_mapped)
        SV_CK(cudaMemcpyAsync(sl.err_host, sl.err_dev, sizeof(int), cudaMemcpyDeviceToHost, sl.stream));
    SV_CK(cudaEventRecord(sl.done, sl.stream));
    return FB_FFT_OK;
}

// Tile prefixes are gathered at the end of the slot's host table while the
// jobs are written, then moved right behind the last job.
int* tile_scratch_of(Slot& sl)
{
    return reinterpret_cast<int*>(sl.tab_host + kBatchJobs * sizeof(PassDesc));
}

// Put the batch on slot sl: its job table (every request's jobs with their
// addresses, grouped by phase and direction, each group with its tile
// prefixes) goes to the device in one copy, then one launch per group, all on
// the slot's stream, between the slot's two events.
int start_batch(fb_fft_server_s* s, Slot& sl)
{
    // jobs first; the tile prefixes go right behind the last job (one copy)
    PassDesc* jobs = reinterpret_cast<PassDesc*>(sl.tab_host);
    int* tiles = tile_scratch_of(sl);
    struct Group {
        bool fwd;
        int job0, njobs, tile0, land, work;
        long long ntiles;
    };
    Group groups[kBatchGroups];
    int ng = 0, nj = 0, nt = 0, phases = 0;
    for (const Req& r : sl.reqs) phases = std::max(phases, r.pe->recipe->phases);
    for (int ph = 0; ph < phases; ++ph) {
        for (int dir = 0; dir < 2; ++dir) {
            const bool fwd = dir == 0;
            Group g{fwd, nj, 0, nt, 16, 16, 0};
            for (size_t i = 0; i < sl.reqs.size(); ++i) {
                const Req& r = sl.reqs[i];
                if ((r.direction == FB_FFT_FORWARD) != fwd) continue;
                char* block = sl.offs[i] >= 0 ? s->arena.base + sl.offs[i] : nullptr;
                const long long scr = up_align(r.pe->recipe->scratch_bytes);
                // host arrays: the transform runs in place in the staging buffer
                const float2* in = r.host_io ? reinterpret_cast<const float2*>(block + scr)
                                             : static_cast<const float2*>(r.in);
                float2* out = r.host_io ? reinterpret_cast<float2*>(block + scr) : static_cast<float2*>(r.out);
                float2* scratch = reinterpret_cast<float2*>(block);
                const bool scale = !fwd && (r.pe->flags & FB_FFT_SCALE_INV_N);
                for (const host::BatchJob& j : r.pe->recipe->jobs) {
                    if (j.phase != ph) continue;
                    PassDesc& d = jobs[nj];
                    d = j.d;
                    d.in = j.src == 0 ? in : (j.src == 1 ? out : scratch);
                    d.out = j.dst == 1 ? out : scratch;
                    d.in_buf = 3;
                    d.out_buf = 3;
                    d.err = sl.err_dev;
                    d.apply_scale = (j.last && scale) ? 1 : 0;
                    tiles[nt++] = (int)g.ntiles;
                    g.ntiles += j.d.ntiles;
                    g.land = std::max(g.land, j.land);
                    g.work = std::max(g.work, j.work);
                    ++nj;
                    ++g.njobs;
                }
            }
            if (g.njobs == 0) {
                nt = g.tile0;
                continue;
            }
            tiles[nt++] = (int)g.ntiles;
            groups[ng++] = g;
        }
    }
    SV_CK(cudaEventRecord(sl.start, sl.stream));
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        const Req& r = sl.reqs[i];
        if (!r.host_io) continue;
        char* stage = s->arena.base + sl.offs[i] + up_align(r.pe->recipe->scratch_bytes);
        SV_CK(cudaMemcpyAsync(stage, r.in, (size_t)r.pe->io, cudaMemcpyHostToDevice, sl.stream));
    }
    int* packed_tiles = reinterpret_cast<int*>(sl.tab_host + (size_t)nj * sizeof(PassDesc));
    std::memmove(packed_tiles, tiles, (size_t)nt * sizeof(int));
    // groups of few jobs carry their tables in the kernel parameter; the
    // table goes to the device only for a larger group
    bool copy = false;
    for (int k = 0; k < ng; ++k) copy = copy || groups[k].njobs > kUnevenInlineJobs;
    if (copy)
        SV_CK(cudaMemcpyAsync(sl.tab_dev, sl.tab_host, (size_t)nj * sizeof(PassDesc) + (size_t)nt * sizeof(int),
                              cudaMemcpyHostToDevice, sl.stream));
    const PassDesc* djobs = reinterpret_cast<const PassDesc*>(sl.tab_dev);
    const int* dtiles = reinterpret_cast<const int*>(sl.tab_dev + (size_t)nj * sizeof(PassDesc));
    for (int k = 0; k < ng; ++k) {
        const Group& g = groups[k];
        const int rc = g.njobs <= kUnevenInlineJobs
                           ? host::batch_launch_inline(g.fwd, jobs + g.job0, packed_tiles + g.tile0, g.njobs,
                                                       g.ntiles, g.land, g.work, sl.stream)
                           : host::batch_launch(g.fwd, djobs + g.job0, dtiles + g.tile0, g.njobs, g.ntiles, g.land,
                                                g.work, sl.stream);
        if (rc != FB_FFT_OK) return rc;
    }
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        const Req& r = sl.reqs[i];
        if (!r.host_io) continue;
        const char* stage = s->arena.base + sl.offs[i] + up_align(r.pe->recipe->scratch_bytes);
        SV_CK(cudaMemcpyAsync(r.out, stage, (size_t)r.pe->io, cudaMemcpyDeviceToHost, sl.stream));
    }
    if (!sl.err_mapped)
        SV_CK(cudaMemcpyAsync(sl.err_host, sl.err_dev, sizeof(int), cudaMemcpyDeviceToHost, sl.stream));
    SV_CK(cudaEventRecord(sl.done, sl.stream));
    s->st.batches++;
    s->st.batched_requests += (long long)sl.reqs.size();
    s->st.largest_batch = std::max(s->st.largest_batch, (long long)sl.reqs.size());
    return FB_FFT_OK;
}

// Move the FIFO head (and, for a batched head, the batched requests right
// behind it that fit the arena and the slot's table) onto slot sl.
// Returns the number moved: 0 when the head's memory is not free yet.
int take_requests(fb_fft_server_s* s, Slot& sl)
{
    const double t = now_s(s);
    int jobs = 0;
    long long tiles = 0;
    while (!s->pending.empty()) {
        Req& r = s->pending.front();
        if (!sl.reqs.empty()) {  // joining a batch
            if (!r.batched || (int)sl.reqs.size() >= s->max_batch) break;
            if (jobs + (int)r.pe->recipe->jobs.size() > kBatchJobs) break;
            if (tiles + r.pe->recipe->tiles >= (1LL << 30)) break;
        }
        long long off = -1;
        if (r.need > 0) {
            off = s->arena.alloc(r.need);
            if (off < 0) break;  // wait for memory (FIFO: no overtaking)
        }
        if (r.batched) {
            jobs += (int)r.pe->recipe->jobs.size();
            tiles += r.pe->recipe->tiles;
        }
        sl.reqs.push_back(r);
        sl.reqs.back().t_admit = t;
        sl.offs.push_back(off);
        s->pending.pop_front();
        s->st.pending--;
        s->st.in_flight++;
        if (!sl.reqs.front().batched) break;  // a per-request head goes alone
    }
    return (int)sl.reqs.size();
}

// Admit FIFO heads while a slot is free and the arena holds the head's needs.
int admit(fb_fft_server_s* s)
{
    while (!s->pending.empty()) {
        int free_slot = -1;
        for (int i = 0; i < (int)s->slots.size(); ++i)
            if (!s->slots[i].busy) {
                free_slot = i;
                break;
            }
        if (free_slot < 0) return FB_FFT_OK;
        Slot& sl = s->slots[free_slot];
        if (take_requests(s, sl) == 0) return FB_FFT_OK;
        sl.busy = true;
        sl.seq = ++s->seq;
        s->busy_slots++;
        s->st.max_in_flight = std::max(s->st.max_in_flight, s->st.in_flight);
        s->st.max_busy_slots = std::max(s->st.max_busy_slots, (long long)s->busy_slots);
        const int rc = sl.reqs.front().batched ? start_batch(s, sl) : start(s, sl, sl.reqs.front(), sl.offs.front());
        if (rc != FB_FFT_OK) {
            // nothing usable was queued behind a failed launch: report it done with the error
            cudaStreamSynchronize(sl.stream);
            cudaGetLastError();
            finish(s, sl, free_slot, rc);
        }
    }
    return FB_FFT_OK;
}

int pump(fb_fft_server_s* s)
{
    int rc = retire(s);
    if (rc != FB_FFT_OK) return rc;
    return admit(s);
}

// Block on the earliest-admitted running request.
int wait_oldest(fb_fft_server_s* s)
{
    Slot* oldest = nullptr;
    for (Slot& sl : s->slots)
        if (sl.busy && (!oldest || sl.seq < oldest->seq)) oldest = &sl;
    if (!oldest) return FB_FFT_OK;
    const cudaError_t e = cudaEventSynchronize(oldest->done);
    if (e != cudaSuccess) cudaGetLastError();  // retire() reports it per request
    return FB_FFT_OK;
}

void free_server(fb_fft_server_s* s)
{
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.start) cudaEventDestroy(sl.start);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.err_host) cudaFreeHost(sl.err_host);
        if (sl.err_dev && !sl.err_mapped) cudaFree(sl.err_dev);
        if (sl.tab_host) cudaFreeHost(sl.tab_host);
        if (sl.tab_dev) cudaFree(sl.tab_dev);
    }
    for (auto& kv : s->plans) {
        host::plan_free(kv.second.plan);
        host::recipe_free(kv.second.recipe);
    }
    if (s->arena.base) cudaFree(s->arena.base);
    if (s->ref) cudaEventDestroy(s->ref);
    if (s->build) cudaStreamDestroy(s->build);
    s->magic = 0;
    delete s;
}

int queue_one(fb_fft_server_s* s, int rank, const long long* dims, long long batch, unsigned flags, int direction,
              const void* in, void* out, int host_io, long long tag);

}  // namespace

extern "C" {

int fb_fft_server_create(fb_fft_server_t* srv, int slots, long long hbm_cap_bytes, int max_plans)
{
    if (!srv) return FB_FFT_ERR_INVALID_ARG;
    *srv = nullptr;
    if (slots < 1 || slots > 64 || hbm_cap_bytes < 0 || max_plans < 1) return FB_FFT_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return FB_FFT_ERR_NO_DEVICE;
    }
    fb_fft_server_s* s = new (std::nothrow) fb_fft_server_s();
    if (!s) return FB_FFT_ERR_ALLOC;
    s->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&s->device);
    s->max_plans = max_plans;
    s->slots.resize(slots);
    s->st.slots = slots;
    int rc = FB_FFT_OK;
    auto ck = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && rc == FB_FFT_OK) rc = host::fail(e, what);
    };
    ck(cudaStreamCreateWithFlags(&s->build, cudaStreamNonBlocking), "cudaStreamCreate");
    ck(cudaEventCreate(&s->ref), "cudaEventCreate");
    if (rc == FB_FFT_OK) {
        ck(cudaEventRecord(s->ref, s->build), "cudaEventRecord");
        ck(cudaEventSynchronize(s->ref), "cudaEventSynchronize");
    }
    // Error words in host memory mapped into the device, where the device's
    // atomics reach host memory natively: the kernels then record a timed-out
    // wait there directly, and no request needs a copy of its error word.
    int native = 0;
    if (cudaDeviceGetAttribute(&native, cudaDevAttrHostNativeAtomicSupported, s->device) != cudaSuccess) {
        cudaGetLastError();
        native = 0;
    }
    for (Slot& sl : s->slots) {
        if (rc != FB_FFT_OK) break;
        ck(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking), "cudaStreamCreate");
        ck(cudaEventCreate(&sl.start), "cudaEventCreate");
        ck(cudaEventCreate(&sl.done), "cudaEventCreate");
        ck(cudaHostAlloc((void**)&sl.tab_host, kTableBytes, cudaHostAllocDefault), "cudaHostAlloc");
        ck(cudaMalloc((void**)&sl.tab_dev, kTableBytes), "cudaMalloc");
        if (native) {
            ck(cudaHostAlloc((void**)&sl.err_host, 16 * sizeof(int), cudaHostAllocMapped), "cudaHostAlloc");
            if (rc == FB_FFT_OK) ck(cudaHostGetDevicePointer((void**)&sl.err_dev, sl.err_host, 0), "cudaHostGetDevicePointer");
            sl.err_mapped = rc == FB_FFT_OK;
            if (rc == FB_FFT_OK) std::memset(sl.err_host, 0, 16 * sizeof(int));
        } else {
            ck(cudaHostAlloc((void**)&sl.err_host, 16 * sizeof(int), cudaHostAllocDefault), "cudaHostAlloc");
            ck(cudaMalloc((void**)&sl.err_dev, 16 * sizeof(int)), "cudaMalloc");
            if (rc == FB_FFT_OK) {
                std::memset(sl.err_host, 0, 16 * sizeof(int));
                ck(cudaMemset(sl.err_dev, 0, 16 * sizeof(int)), "cudaMemset");
            }
        }
    }
    if (rc == FB_FFT_OK && hbm_cap_bytes > 0) {
        const long long cap = hbm_cap_bytes / kArenaAlign * kArenaAlign;
        if (cudaMalloc((void**)&s->arena.base, (size_t)cap) != cudaSuccess) {
            cudaGetLastError();
            s->arena.base = nullptr;
            rc = FB_FFT_ERR_ALLOC;
        } else {
            s->arena.reset(cap);
        }
    }
    if (rc != FB_FFT_OK) {
        free_server(s);
        return rc;
    }
    s->st.arena_bytes = s->arena.cap;
    *srv = s;
    return FB_FFT_OK;
}

int fb_fft_server_prepare(fb_fft_server_t srv, int rank, const long long* dims, long long batch, unsigned flags)
{
    if (!server_ok(srv)) return FB_FFT_ERR_BAD_PLAN;
    PlanEntry* pe = nullptr;
    const int rc = get_plan(srv, rank, dims, batch, flags, &pe);
    if (rc == FB_FFT_OK) evict_idle(srv);
    return rc;
}

int fb_fft_server_submit(fb_fft_server_t srv, int rank, const long long* dims, long long batch, unsigned flags,
                         int direction, const void* in, void* out, int host_io, long long tag)
{
    if (!server_ok(srv)) return FB_FFT_ERR_BAD_PLAN;
    const int rc = queue_one(srv, rank, dims, batch, flags, direction, in, out, host_io, tag);
    if (rc != FB_FFT_OK) return rc;
    return pump(srv);
}

int fb_fft_server_submit_many(fb_fft_server_t srv, const fb_fft_server_request* reqs, int count, int* status)
{
    if (!server_ok(srv)) return FB_FFT_ERR_BAD_PLAN;
    if (count < 0 || (count > 0 && (!reqs || !status))) return FB_FFT_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        const fb_fft_server_request& q = reqs[i];
        status[i] = queue_one(srv, q.rank, q.dims, q.batch, q.flags, q.direction, q.in, q.out, q.host_io, q.tag);
    }
    return pump(srv);
}

}  // extern "C"

namespace {

// Validate one request and append it to the FIFO (no admission).
int queue_one(fb_fft_server_s* s, int rank, const long long* dims, long long batch, unsigned flags, int direction,
              const void* in, void* out, int host_io, long long tag)
{
    if (direction != FB_FFT_FORWARD && direction != FB_FFT_INVERSE) {
        s->st.rejected++;
        return FB_FFT_ERR_INVALID_ARG;
    }
    PlanEntry* pe = nullptr;
    int rc = get_plan(s, rank, dims, batch, flags, &pe);
    if (rc == FB_FFT_OK && pe->io > 0) {
        if (!in || !out) rc = FB_FFT_ERR_INVALID_ARG;
        const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out, n = (uintptr_t)pe->io;
        if (!host_io && ((a | b) & 7)) rc = FB_FFT_ERR_INVALID_ARG;
        if (!host_io && a != b && a < b + n && b < a + n) rc = FB_FFT_ERR_INVALID_ARG;
    }
    Req r;
    if (rc == FB_FFT_OK) {
        r.batched = pe->recipe != nullptr && s->max_batch > 1;
        r.need = request_need(pe, host_io != 0, r.batched);
        if (r.need > s->arena.cap) rc = FB_FFT_ERR_OVER_BUDGET;
    }
    if (rc != FB_FFT_OK) {
        s->st.rejected++;
        evict_idle(s);
        return rc;
    }
    r.tag = tag;
    r.pe = pe;
    r.direction = direction;
    r.in = in;
    r.out = out;
    r.host_io = host_io != 0;
    r.t_submit = now_s(s);
    pe->users++;
    s->pending.push_back(r);
    s->st.submitted++;
    s->st.pending++;
    evict_idle(s);
    return FB_FFT_OK;
}

}  // namespace

extern "C" {

int fb_fft_server_poll(fb_fft_server_t srv, int wait, fb_fft_server_done* done, int capacity, int* n_done)
{
    if (!server_ok(srv)) return FB_FFT_ERR_BAD_PLAN;
    if (!n_done || capacity < 0 || (capacity > 0 && !done)) return FB_FFT_ERR_INVALID_ARG;
    fb_fft_server_s* s = srv;
    int rc = pump(s);
    if (rc != FB_FFT_OK) return rc;
    if (wait && s->done.empty() && s->st.in_flight > 0) {
        wait_oldest(s);
        rc = pump(s);
        if (rc != FB_FFT_OK) return rc;
    }
    int n = 0;
    while (n < capacity && !s->done.empty()) {
        done[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_done = n;
    return FB_FFT_OK;
}

int fb_fft_server_drain(fb_fft_server_t srv)
{
    if (!server_ok(srv)) return FB_FFT_ERR_BAD_PLAN;
    fb_fft_server_s* s = srv;
    for (;;) {
        int rc = pump(s);
        if (rc != FB_FFT_OK) return rc;
        if (s->st.in_flight == 0) {
            if (s->pending.empty()) return FB_FFT_OK;
            // a queued head that cannot be admitted with every slot idle never will be
            return FB_FFT_ERR_OVER_BUDGET;
        }
        wait_oldest(s);
    }
}

int fb_fft_server_cancel(fb_fft_server_t srv, long long tag)
{
    if (!server_ok(srv)) return FB_FFT_ERR_BAD_PLAN;
    fb_fft_server_s* s = srv;
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
        if (it->tag != tag) continue;
        fb_fft_server_done d;
        d.tag = tag;
        d.status = FB_FFT_ERR_CANCELLED;
        d.slot = -1;
        d.t_submit = it->t_submit;
        d.t_admit = -1.0;
        d.t_done = now_s(s);
        d.t_dev_start = d.t_dev_end = -1.0;
        it->pe->users--;
        s->pending.erase(it);
        s->done.push_back(d);
        s->st.pending--;
        s->st.cancelled++;
        return pump(s);
    }
    return FB_FFT_ERR_INVALID_ARG;
}

int fb_fft_server_wait(fb_fft_server_t srv, double until_s)
{
    if (!server_ok(srv)) return FB_FFT_ERR_BAD_PLAN;
    fb_fft_server_s* s = srv;
    for (;;) {
        const int rc = pump(s);
        if (rc != FB_FFT_OK) return rc;
        if (!s->done.empty() || s->st.in_flight == 0 || now_s(s) >= until_s) return FB_FFT_OK;
    }
}

int fb_fft_server_set_batch(fb_fft_server_t srv, int max_requests)
{
    if (!server_ok(srv)) return FB_FFT_ERR_BAD_PLAN;
    srv->max_batch = max_requests < 1 ? 1 : max_requests;
    return FB_FFT_OK;
}

double fb_fft_server_clock(fb_fft_server_t srv) { return server_ok(srv) ? now_s(srv) : -1.0; }

int fb_fft_server_stats_get(fb_fft_server_t srv, fb_fft_server_stats* stats)
{
    if (!server_ok(srv)) return FB_FFT_ERR_BAD_PLAN;
    if (!stats) return FB_FFT_ERR_INVALID_ARG;
    fb_fft_server_s* s = srv;
    s->st.plans = (long long)s->plans.size();
    s->st.arena_in_use = s->arena.used;
    s->st.arena_peak = s->arena.peak;
    *stats = s->st;
    return FB_FFT_OK;
}

int fb_fft_server_destroy(fb_fft_server_t srv)
{
    if (!srv) return FB_FFT_OK;
    if (!server_ok(srv)) return FB_FFT_ERR_BAD_PLAN;
    free_server(srv);
    return FB_FFT_OK;
}

}  // extern "C"
