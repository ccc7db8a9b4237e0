/*
 * fb_fft.h -- C ABI of the GB300 complex FFT function block.
 *
 * The paper (Sec. 3.3, Sec. 3.4 C-1/C-2) offloads a whole "function block" of
 * a C application -- its example is the Fourier transform, Sec. 5.1(a) --
 * by deleting the CPU code and calling a device implementation through an
 * interface that matches the host program's call: the array, its dimensions,
 * the direction, in place or not.  This header is that interface for the
 * complex-to-complex DFT, implemented from scratch for sm_103a:
 *
 *     X[k] = c * sum_{n=0}^{N-1} x[n] * exp(s * 2*pi*i * n*k / N)
 *
 * (the textbook DFT; the paper itself defers the formula to the library it
 * swaps in, Sec. 5.1(a)), with exponent sign s = `direction`, c = 1 unless
 * FB_FFT_SCALE_INV_N asks for 1/N on inverse transforms, applied along every
 * axis of a rank-1..3 array and independently for each batch item.
 *
 * Data layout (all entry points): complex64 interleaved {float re, float im},
 * row-major, last dimension fastest, batch items contiguous one after
 * another (batch stride = prod(dims) elements).  Every call returns an
 * fb_fft_status value; on an argument error no output is touched.
 *
 * Thread safety: distinct plans may be used from distinct host threads; one
 * plan must not be executed concurrently from two threads.
 */
#ifndef FB_FFT_H
#define FB_FFT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fb_fft_plan_s* fb_fft_plan_t;

typedef enum fb_fft_status {
    FB_FFT_OK = 0,
    FB_FFT_ERR_INVALID_ARG = -1,      /* null pointer, bad rank/dim/direction, misaligned */
    FB_FFT_ERR_UNSUPPORTED_SIZE = -2, /* a dim is not 2^a*3^b*5^c or exceeds the limits */
    FB_FFT_ERR_ALLOC = -3,            /* device or host allocation failed */
    FB_FFT_ERR_CUDA = -4,             /* a CUDA runtime call or kernel launch failed */
    FB_FFT_ERR_TIMEOUT = -5,          /* a bounded device-side wait gave up */
    FB_FFT_ERR_BAD_PLAN = -6,         /* null or destroyed plan handle */
    FB_FFT_ERR_NO_DEVICE = -7,        /* no CUDA device is visible */
    FB_FFT_ERR_CANCELLED = -8,        /* a server request was cancelled before it ran */
    FB_FFT_ERR_OVER_BUDGET = -9       /* a server request can never fit the device-memory budget */
} fb_fft_status;

/* Exponent sign of the transform kernel exp(s*2*pi*i*n*k/N). */
#define FB_FFT_FORWARD (-1)
#define FB_FFT_INVERSE (+1)

/* Plan flags. */
#define FB_FFT_SCALE_INV_N 0x1u /* multiply the result of every INVERSE exec by 1/prod(dims) */
/* The same transform (Sec. 5.1(a); the paper fixes no arithmetic precision)
 * with the radix-16 stages of power-of-two lines of length >= 256 on the
 * tensor cores: each stage's 16-point DFT as one FP16 matrix product per 128
 * butterflies, inputs and DFT matrix split into hi + lo halves (three
 * products, FP32 accumulation, per-butterfly power-of-two scaling).  Relative
 * L2 error per result <= 5e-5 (the FP32 path: <= 2e-6 log2 N).  Other stages
 * and other lengths run the FP32 butterflies.  Not for fb_fft_plan_many. */
#define FB_FFT_TENSOR_CORES 0x2u

/* Largest supported length along one axis of a rank-2/3 plan, and of a
 * rank-1 plan (a rank-1 length above FB_FFT_MAX_SMEM_LEN runs as a two-pass
 * "four-step" transform, N = N1 * N2). */
#define FB_FFT_MAX_SMEM_LEN 4096LL
#define FB_FFT_MAX_1D_LEN (4096LL * 4096LL)

/*
 * fb_fft_plan -- prepare a transform (Sec. 3.4 C-1: the replaced block is
 * connected once, then called like the CPU routine it replaces).
 *   plan   out: new handle, owned by the caller until fb_fft_destroy.
 *   rank   1, 2 or 3.
 *   dims   rank lengths, row-major (dims[rank-1] is contiguous); each >= 1
 *          and 5-smooth (2^a 3^b 5^c); <= FB_FFT_MAX_SMEM_LEN for rank >= 2,
 *          <= FB_FFT_MAX_1D_LEN for rank 1.
 *   batch  number of transforms (>= 0) laid out back to back.
 *   flags  0 or FB_FFT_SCALE_INV_N and/or FB_FFT_TENSOR_CORES.
 *   stream cudaStream_t the plan launches on (NULL = legacy default stream).
 * Builds the twiddle tables on the GPU (FP64 evaluation, rounded to FP32) and
 * allocates the plan's scratch; both are owned by the plan.  Uses the current
 * CUDA device; the plan must later be used with that device current.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, ALLOC, CUDA, NO_DEVICE.
 */
int fb_fft_plan(fb_fft_plan_t* plan, int rank, const long long* dims, long long batch,
                unsigned flags, void* stream);

/*
 * Batched uneven lengths (the paper's block offload applied to many calls at
 * once, Sec. 3.4 C-1 / Sec. 3.3: one replaced block serving a workload of
 * transforms of different sizes).
 *
 * fb_fft_many_layout -- the packed layout such a plan expects: transform i
 * (length lengths[i]) starts at element offsets[i] = sum over j < i of
 * lengths[j] rounded up to even (every transform 16-byte aligned).  Writes
 * offsets (if not NULL) and returns the total element count, or -1 on bad
 * arguments.  Host only.
 *
 * fb_fft_plan_many -- plan `count` 1-D transforms of the given 5-smooth
 * lengths (each <= FB_FFT_MAX_1D_LEN) laid out as above; fb_fft_exec /
 * fb_fft_exec_host then take buffers of fb_fft_many_layout(...) elements.
 * Transforms of one length run as one pass through an offset table (long
 * ones as a four-step pair).  By default (engine 0 below) every pass of the
 * batch is one persistent kernel launch; otherwise different lengths run
 * concurrently on plan-owned side streams.  Each exec is replayed as one
 * CUDA graph launch (captured on the first exec with a given
 * in/out/direction).  One exec of a plan at a time: the plan's device
 * counters and scratch serve one exec.
 * FB_FFT_SCALE_INV_N scales each inverse result by 1/its length.
 * Errors: as fb_fft_plan.
 *
 * fb_fft_set_graph -- 0 launches the passes directly instead of through the
 * graph (same results; used to compare the two).
 */
long long fb_fft_many_layout(int count, const long long* lengths, long long* offsets);
int fb_fft_plan_many(fb_fft_plan_t* plan, int count, const long long* lengths, unsigned flags, void* stream);
int fb_fft_set_graph(fb_fft_plan_t plan, int enable);

/*
 * Tuning knobs of a batched uneven plan (all 0 = the defaults):
 *   streams            side streams the length groups spread over (1..32; default 4)
 *   use_graph          1/0: replay one CUDA graph per exec (default) / launch directly;
 *                      any other value = default
 *   chunk_bytes        four-step intermediate per chunk of a length group (default 512 MiB)
 *   odd_radices_first  lengths with factors 3/5 (generic kernel): 1 runs the 5s and 3s
 *                      before the power-of-two radices
 *   max_lines          generic kernel: at most this many lines per tile (0 = no extra cap)
 *   engine             0 (default): one kernel for every pass, ONE launch per
 *                      exec over a device job table (each job one length group
 *                      or four-step chunk, lines up to 2048 points; longer
 *                      lengths split into two such jobs): CTAs claim tiles in
 *                      table order from a device counter, and a four-step row
 *                      tile waits (bounded) until its chunk's column tiles are
 *                      done.  Taken whenever every length fits it, else
 *                      engine 1.
 *                      2: the same kernel in two launches per exec (all single
 *                      passes and four-step columns, then all rows; the same
 *                      results), when every length fits it, else engine 1.
 *                      1: the per-kernel schedule below (side streams, CUDA graph).
 *   per_length         engine 1: one launch per length group for every kernel
 *                      (1), or (0, default) passes of lengths with a factor 3 or 5
 *                      that share a power-of-two factor run as one launch (up to
 *                      64 lengths each), four-step groups with disjoint scratch, in
 *                      two phases (single passes and four-step columns, then
 *                      four-step rows).  per_length = 1 selects engine 1.
 *   streams, use_graph, odd_radices_first, max_lines: engine 1 only.
 */
typedef struct fb_fft_many_opts {
    int streams;
    int use_graph;
    long long chunk_bytes;
    int odd_radices_first;
    int max_lines;
    int per_length;
    int engine;
} fb_fft_many_opts;
int fb_fft_plan_many_ex(fb_fft_plan_t* plan, int count, const long long* lengths, unsigned flags, void* stream,
                        const fb_fft_many_opts* opts);

/*
 * fb_fft_autotune_many -- the project's autotuner for batched uneven plans
 * (the paper's verification step, Sec. 3.4 / Sec. 4.2: measure candidate
 * offload patterns in the target environment, keep the fastest).  Plans,
 * runs and times (CUDA events, `reps` execs after two warm-ups) candidate
 * settings -- engine 0 with each chunk_bytes, engine 2 at the best of them,
 * then engine 1 by coordinate
 * descent over streams, chunk_bytes, odd_radices_first, max_lines and
 * per_length -- on the caller's device buffers `in`/`out`
 * (layout of fb_fft_many_layout; `out` is overwritten) in `direction`,
 * and writes the fastest settings to *best and their time per exec (ms)
 * to *best_ms.  Synchronous.  Errors: as fb_fft_plan_many / fb_fft_exec.
 */
int fb_fft_autotune_many(int count, const long long* lengths, unsigned flags, const void* in, void* out,
                         int direction, void* stream, int reps, fb_fft_many_opts* best, float* best_ms);

/*
 * fb_fft_exec -- run the transform on device buffers (Sec. 3.3 / Sec. 5.1(a):
 * the Fourier transform block itself).
 *   in        device pointer to batch*prod(dims) complex64 values, 8-byte aligned.
 *   out       device pointer of the same size; out == in transforms in place.
 *             Partial overlap of in and out is an INVALID_ARG.
 *   direction FB_FFT_FORWARD or FB_FFT_INVERSE (the exponent sign).
 * Asynchronous: enqueued on the plan's stream, no host synchronisation.
 * `in` is read only (never clobbered) when out != in.  The caller keeps
 * ownership of both buffers.  Errors: BAD_PLAN, INVALID_ARG, CUDA.
 */
int fb_fft_exec(fb_fft_plan_t plan, const void* in, void* out, int direction);

/*
 * fb_fft_exec_host -- the drop-in form of the replaced CPU call (Sec. 3.4
 * C-1, Sec. 5.1(b)): host arrays in and out.  Copies host_in to a
 * plan-owned device buffer, transforms, copies the result to host_out and
 * waits for it.  host_in/host_out may be the same array (in place) and may be
 * pageable or pinned host memory.  The first call allocates the device
 * staging buffer (owned by the plan).  With pinned arrays and a batch of at
 * least two 32 MiB chunks, the batch moves in chunks whose copy in,
 * transform and copy out overlap (plan-owned copy streams and chunk plans,
 * created on first use; same results); FB_FFT_HOST_PIPELINE=0 turns this off.
 * Errors: BAD_PLAN, INVALID_ARG, ALLOC, CUDA, TIMEOUT.
 */
int fb_fft_exec_host(fb_fft_plan_t plan, const void* host_in, void* host_out, int direction);

/*
 * fb_fft_check -- wait for the plan's stream and report whether any kernel of
 * this plan gave up on a bounded device-side wait since the last check
 * (FB_FFT_ERR_TIMEOUT; the word is then cleared).  exec_host calls it.
 */
int fb_fft_check(fb_fft_plan_t plan);

/*
 * fb_fft_debug_inject_timeout -- test hook for the failure path.  While
 * enabled, every TMA-fed kernel of this plan announces 16 more bytes per tile
 * than it copies, so its bounded wait runs out (after about one second),
 * the kernel records the error and returns early, and the next fb_fft_check
 * reports FB_FFT_ERR_TIMEOUT.  In a one-launch batched uneven exec every
 * four-step row's dependency target is raised out of reach instead: the
 * first wait to run out (after about a second) ends the others, the tiles
 * run on, and the check reports the same error.  Nothing faults and the context stays usable;
 * the output of such an exec is undefined.  Not for production use.
 */
int fb_fft_debug_inject_timeout(fb_fft_plan_t plan, int enable);

/*
 * fb_fft_offload_decide -- the paper's verification step for one function
 * block (Sec. 3.4 / Sec. 4.2: each replaceable block is measured offloaded
 * and not offloaded in the verification environment, and offloaded only if
 * that is faster).  Times `reps` calls of the caller's own CPU routine
 * cpu(ctx, host_in, host_out, direction) against `reps` calls of
 * fb_fft_exec_host(plan, host_in, host_out, direction) (host->device copy,
 * transform, device->host copy), after one untimed call of each, with a
 * monotonic host clock; writes the mean times per call and *use_gpu = 1 when
 * the device path is faster.  host_out is overwritten.  The library never
 * runs a CPU transform of its own: `cpu` is the caller's block.
 * Errors: BAD_PLAN, INVALID_ARG, and those of fb_fft_exec_host.
 */
typedef void (*fb_fft_cpu_block)(void* ctx, const void* host_in, void* host_out, int direction);
int fb_fft_offload_decide(fb_fft_plan_t plan, fb_fft_cpu_block cpu, void* ctx, const void* host_in, void* host_out,
                          int direction, int reps, int* use_gpu, double* cpu_ms, double* gpu_ms);

/* fb_fft_set_stream -- change the stream later execs launch on. */
int fb_fft_set_stream(fb_fft_plan_t plan, void* stream);

/* fb_fft_destroy -- free the plan and everything it owns; NULL is a no-op.
 * Synchronises the plan's stream first. */
int fb_fft_destroy(fb_fft_plan_t plan);

/* fb_fft_status_string -- static English text for a status code. */
const char* fb_fft_status_string(int status);

/* fb_fft_last_error -- the CUDA call that last failed on this host thread and
 * CUDA's text for it ("" if none); valid until this thread's next failure. */
const char* fb_fft_last_error(void);

/*
 * Plan description (host-side facts of the schedule).
 *   passes         kernel launches per exec
 *   tc_passes      of which with radix-16 stages on the tensor cores
 *   smem_len_max   longest line held in one CTA's shared memory
 *   scratch_bytes  plan-owned device scratch (four-step intermediate)
 *   twiddle_bytes  plan-owned device twiddle tables
 *   elements       prod(dims);  batch  as planned
 */
typedef struct fb_fft_info {
    int passes;
    int tc_passes;
    long long smem_len_max;
    long long scratch_bytes;
    long long twiddle_bytes;
    long long elements;
    long long batch;
} fb_fft_info;
int fb_fft_plan_info(fb_fft_plan_t plan, fb_fft_info* info);

/*
 * fb_fft_plan_query -- run the planner on the host only (no device, no
 * allocation) and describe the plan fb_fft_plan would build for these
 * arguments.  Same errors as fb_fft_plan except ALLOC/CUDA/NO_DEVICE.
 */
int fb_fft_plan_query(int rank, const long long* dims, long long batch, unsigned flags, fb_fft_info* info);

/* fb_fft_plan_many_query -- the same for fb_fft_plan_many (host only). */
int fb_fft_plan_many_query(int count, const long long* lengths, unsigned flags, fb_fft_info* info);

/*
 * fb_fft_factorize -- the planner's radix schedule for one in-shared-memory
 * line length n (host only, needs no GPU).  Writes the radices (each of
 * 2,3,4,5,8,16, product n) to radices[0..*count).  Errors: INVALID_ARG,
 * UNSUPPORTED_SIZE (n not 5-smooth or > FB_FFT_MAX_SMEM_LEN).
 */
int fb_fft_factorize(long long n, int* radices, int capacity, int* count);

/*
 * fb_fft_split -- the planner's four-step split of a rank-1 length n
 * (host only): n = *n1 * *n2 with n1, n2 <= FB_FFT_MAX_SMEM_LEN; *n1 = n,
 * *n2 = 1 when n fits one pass.  Errors: INVALID_ARG, UNSUPPORTED_SIZE.
 */
int fb_fft_split(long long n, long long* n1, long long* n2);

/*
 * Profiling.  fb_fft_profile(plan, 1) makes every later exec record a CUDA
 * event pair around each of its kernel launches (on the plan's stream);
 * fb_fft_profile_read synchronises on them, writes per-pass totals
 * (ms_total[p], launches[p], p < *npasses, at most `capacity`) and clears the
 * record.  Events are cheap but not free; leave profiling off in production.
 */
int fb_fft_profile(fb_fft_plan_t plan, int enable);
int fb_fft_profile_read(fb_fft_plan_t plan, double* ms_total, long long* launches,
                        int capacity, int* npasses);

/* fb_fft_pass_launch -- (introspection, no paper counterpart) launch
 * configuration of the plan's pass p, in plan
 * order (fb_fft_info.passes of them for regular plans): CTAs, threads per
 * CTA, dynamic shared memory in bytes (with TMA on).  A batched-uneven pass
 * that runs inside a merged launch reports grid 0.  Errors: BAD_PLAN,
 * INVALID_ARG. */
int fb_fft_pass_launch(fb_fft_plan_t plan, int pass, long long* grid, int* block, long long* smem_bytes);

/* Name of the kernel pass p launches (static string), or NULL. */
const char* fb_fft_pass_name(fb_fft_plan_t plan, int pass);

/* Total kernels this library has launched in this process (all plans). */
long long fb_fft_launch_count(void);

/*
 * fb_fft_twiddles -- evaluate exp(-2*pi*i*m/d) for m = 0..count-1 with the
 * library's twiddle kernel (FP64 on the GPU, rounded to FP32) and copy the
 * float pairs to host_out[2*count].  Exposed so tests can check the tables.
 * Errors: INVALID_ARG, ALLOC, CUDA, NO_DEVICE.
 */
int fb_fft_twiddles(long long d, long long count, float* host_out);

/*
 * Serving: continuous batching of offload calls.
 *
 * The paper replaces a function block of an application that keeps running
 * in its production environment (Sec. 3.1, Sec. 5.1(c)); when many callers
 * offload transforms of mixed shapes to one GPU, calling fb_fft_plan/exec per
 * call serialises them.  A server keeps plans resident (one per shape, shared
 * by all slots: twiddle tables are read-only) and runs each admitted request,
 * or batch of queued requests (fb_fft_server_set_batch), on one of `slots`
 * CUDA streams, so the copies and kernels of requests that arrive while
 * others run overlap on the device.  A request is admitted, in
 * arrival (FIFO) order, as soon as a slot is free and its device bytes fit in
 * the server's memory budget: an arena of `hbm_cap_bytes` reserved once at
 * creation, from which each request takes its four-step scratch and, for
 * host-array requests, one staging buffer; both return to the arena when the
 * request completes.  Completion is observed with a CUDA event per slot; every
 * submit and poll first retires finished requests and admits waiting ones;
 * slots never wait for one another (the requests of one batch are reported
 * done together).  Nothing blocks except poll with wait != 0 and drain.
 *
 * Not thread-safe: one host thread drives a server.  The device current at
 * fb_fft_server_create must be current on every later call.
 */
typedef struct fb_fft_server_s* fb_fft_server_t;

/* One finished request.  Times are seconds on the server's monotonic clock
 * (fb_fft_server_clock): t_submit at fb_fft_server_submit, t_admit when it
 * went to a slot, t_done when a submit/poll/drain saw its completion event.
 * t_dev_start / t_dev_end: when the request's work began and ended on the
 * device (CUDA event timestamps on its slot's stream, seconds after an
 * event the server recorded at creation), -1 when it did not run or failed;
 * requests on different slots whose device intervals intersect overlapped
 * on the GPU. */
typedef struct fb_fft_server_done {
    long long tag;     /* the caller's tag from submit */
    int status;        /* FB_FFT_OK, FB_FFT_ERR_CANCELLED, _TIMEOUT or _CUDA */
    int slot;          /* stream slot it ran on, -1 if it never ran */
    double t_submit, t_admit, t_done;
    double t_dev_start, t_dev_end;
} fb_fft_server_done;

typedef struct fb_fft_server_stats {
    long long submitted, completed, rejected, cancelled;
    long long pending, in_flight;          /* now */
    long long plans, plan_builds, plan_bytes; /* resident plans, plans built, their device bytes */
    long long arena_bytes, arena_in_use, arena_peak;
    long long max_in_flight;               /* most requests admitted and not yet retired at once */
    int slots;
    int reserved;
    long long batches;                     /* batches run (see fb_fft_server_set_batch) */
    long long batched_requests;            /* requests that ran in them */
    long long largest_batch;               /* most requests in one batch */
    long long max_busy_slots;              /* most slots busy at once (<= slots) */
} fb_fft_server_stats;

/*
 * fb_fft_server_create
 *   srv            out: new handle, owned by the caller until fb_fft_server_destroy.
 *   slots          1..64 concurrent requests (one CUDA stream each).
 *   hbm_cap_bytes  >= 0: device bytes the server may hold for requests (one
 *                  cudaMalloc at creation; 0 admits only requests that need
 *                  no scratch and no staging).
 *   max_plans      >= 1: resident plans kept; the least recently used idle
 *                  plan is freed beyond that.
 * Errors: INVALID_ARG, ALLOC, CUDA, NO_DEVICE.
 */
int fb_fft_server_create(fb_fft_server_t* srv, int slots, long long hbm_cap_bytes, int max_plans);

/*
 * fb_fft_server_set_batch -- how many queued requests one slot may take at
 * once (default 64: with 8 slots, batches of 64 keep several slots' batches
 * overlapping on the device; larger ones leave fewer, longer batches).  A shape whose every axis (or, for a 1-D length above
 * 2048, both four-step factors) is at most 2048 points and that does not ask
 * for the tensor cores has a resident batch recipe; when a slot frees up, the
 * queue's head and the recipe requests right behind it (FIFO, as long as
 * the memory budget holds them, at most max_requests and 1024 jobs) run
 * together: their job descriptors, with each request's own addresses, go to
 * the device in one copy and run as one launch per phase and direction (at
 * most six launches for the whole batch).  The batch grows with the queue:
 * a request that finds a slot free starts at once, alone.  Results do not
 * depend on what else is in the batch (same bits alone and in any batch);
 * they can differ in the last bits from the per-request path, which uses the
 * plan's own kernels.
 *   max_requests  <= 1: no batching, every request runs alone through its
 *                 shape's plan (the per-call kernels).  Applies to requests
 *                 submitted after the call.
 * Errors: BAD_PLAN.
 */
int fb_fft_server_set_batch(fb_fft_server_t srv, int max_requests);

/*
 * fb_fft_server_submit -- queue one transform (rank, dims, batch, flags as
 * fb_fft_plan; direction as fb_fft_exec).
 *   in, out   host_io == 0: device pointers (8-byte aligned, equal or not
 *             overlapping), owned by the caller and untouched by the caller
 *             until the request is reported done.
 *             host_io != 0: host pointers (pinned memory gives asynchronous
 *             copies; in == out is allowed); the server copies through an
 *             arena staging buffer.
 *   tag       caller's identifier, reported back by poll.
 * A plan for a new shape is built here, synchronously (charged to this call;
 * create plans ahead with fb_fft_server_prepare).  Returns OK when queued;
 * OVER_BUDGET when the request needs more than the whole arena; the plan
 * errors (INVALID_ARG, UNSUPPORTED_SIZE, ALLOC, CUDA) otherwise.  A rejected
 * request is counted in stats.rejected and never reported by poll.
 */
int fb_fft_server_submit(fb_fft_server_t srv, int rank, const long long* dims, long long batch, unsigned flags,
                         int direction, const void* in, void* out, int host_io, long long tag);

/* One request of fb_fft_server_submit_many: the arguments of
 * fb_fft_server_submit (dims[rank..2] are ignored). */
typedef struct fb_fft_server_request {
    long long dims[3];
    long long batch;
    long long tag;
    const void* in;
    void* out;
    int rank;
    unsigned flags;
    int direction;
    int host_io;
} fb_fft_server_request;

/*
 * fb_fft_server_submit_many -- queue `count` requests in this order, then
 * admit once: what a caller holding several requests that arrived together
 * hands over in one call, so that the queue they form can run as one batch
 * (fb_fft_server_set_batch) instead of each being admitted while the next
 * is still being submitted.  status[i] receives what fb_fft_server_submit
 * would return for reqs[i] (a rejected request is not queued; the others
 * still are).  reqs and status: `count` entries, owned by the caller, not
 * kept after the call.
 * Errors (nothing queued): BAD_PLAN, INVALID_ARG (count < 0, or a null
 * array with count > 0); CUDA from the admission.
 */
int fb_fft_server_submit_many(fb_fft_server_t srv, const fb_fft_server_request* reqs, int count, int* status);

/* fb_fft_server_prepare -- build (or touch) the resident plan of a shape now. */
int fb_fft_server_prepare(fb_fft_server_t srv, int rank, const long long* dims, long long batch, unsigned flags);

/*
 * fb_fft_server_poll -- retire finished requests, admit waiting ones, then
 * move up to `capacity` finished requests (oldest first) into done[] and set
 * *n_done.  wait != 0 and nothing finished yet: block until the oldest request
 * on a slot completes (returns at once when nothing is queued or running).
 * Errors: INVALID_ARG, CUDA.
 */
int fb_fft_server_poll(fb_fft_server_t srv, int wait, fb_fft_server_done* done, int capacity, int* n_done);

/*
 * fb_fft_server_wait -- retire and admit (as poll does) until a request has
 * finished, nothing is running, or the server clock (fb_fft_server_clock)
 * reaches until_s, whichever comes first; finished requests stay for poll.
 * For a caller that has nothing to submit before until_s (its next
 * arrival): completions are seen as they happen, not at the caller's next
 * poll.  It spins on the host (no sleep).  Errors: BAD_PLAN, CUDA.
 */
int fb_fft_server_wait(fb_fft_server_t srv, double until_s);

/* fb_fft_server_drain -- block until nothing is queued or running; finished
 * requests stay available to poll. */
int fb_fft_server_drain(fb_fft_server_t srv);

/* fb_fft_server_cancel -- drop a queued (not yet admitted) request; poll then
 * reports it with FB_FFT_ERR_CANCELLED.  A request already on a slot cannot be
 * cancelled: INVALID_ARG, as for an unknown tag. */
int fb_fft_server_cancel(fb_fft_server_t srv, long long tag);

/* fb_fft_server_clock -- seconds since the server was created (the clock of
 * fb_fft_server_done), or -1 for a bad handle. */
double fb_fft_server_clock(fb_fft_server_t srv);

int fb_fft_server_stats_get(fb_fft_server_t srv, fb_fft_server_stats* stats);

/* fb_fft_server_destroy -- wait for running requests, drop queued ones, free
 * plans, arena and streams; NULL is a no-op. */
int fb_fft_server_destroy(fb_fft_server_t srv);

/*
 * fb_fft_exec_1d_noalloc -- batched 1-D transform that allocates no device
 * memory.  The paper has no counterpart.  It is for callers that cannot call
 * cudaMalloc: a plug-in or embedded library whose host application owns all
 * device memory through its own allocator (and may forbid driver
 * allocations), real-time code that must not enter an allocator that can
 * block, or code that must run in a device-memory budget fixed in advance.
 * For them fb_fft_plan's device-resident twiddle tables and scratch are not
 * an option.
 *   in, out    device pointers, batch*n complex64 values each, 8-byte aligned;
 *              out == in runs in place, partial overlap is INVALID_ARG.
 *   n          5-smooth length, 1 <= n <= 4194304 (2^22) and splittable as the
 *              plan API's four-step (fb_fft_split); larger n is
 *              FB_FFT_ERR_UNSUPPORTED_SIZE.  n = 1 is a copy.
 *   batch      >= 0 transforms back to back (any count: they run in chunks).
 *   direction  FB_FFT_FORWARD / FB_FFT_INVERSE.
 *   flags      0, FB_FFT_SCALE_INV_N, and/or FB_FFT_NOALLOC_CHECK: wait for
 *              the transform to finish (synchronises `stream`) and return
 *              FB_FFT_ERR_TIMEOUT if one of its device-side waits gave up.
 *              Without it the call returns once the work is enqueued and
 *              a timed-out wait goes unreported.
 *   stream     cudaStream_t (NULL = legacy default stream).
 * Runs the same kernels, tiles and four-step split as fb_fft_plan for this
 * length, asynchronously on `stream`.  Twiddle tables, the four-step
 * intermediate and the error word live in one file-scope device array of the
 * library (32 MiB + 256 KiB + 256 bytes, held by every GPU that loads the
 * library until the process exits).  The first call on each device looks up
 * that array's device address (cudaGetSymbolAddress) with the device current.
 * Every call reuses and overwrites the array: calls that overlap on the GPU
 * race, so serialise them (one stream, or events).  The first launch of each
 * kernel in the process also sets its shared-memory limit.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, CUDA, TIMEOUT (with the check flag).
 */
#define FB_FFT_NOALLOC_CHECK 0x100u
int fb_fft_exec_1d_noalloc(const void* in, void* out, long long n, long long batch, int direction,
                           unsigned flags, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FB_FFT_H */
