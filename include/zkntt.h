/*
 * zkntt.h -- C ABI of the GB300 (sm_103a) number-theoretic transform library.
 *
 * The transform (arxiv 2509.22684, Section II-B): for a vector a_0..a_{n-1} of
 * elements of a prime field F_r and a primitive n-th root of unity w,
 *     A_k = sum_{j=0}^{n-1} a_j * w^(j*k)        (k = 0..n-1, n = 2^log_n).
 * The inverse uses w^-1 and multiplies by n^-1, so inverse(forward(a)) = a
 * (the paper treats NTT and INTT as the same computation, Section II-B).
 * A coset transform with shift g (Groth16 prover, Fig. 2) is
 *     forward:  A_k = sum_j (a_j g^j) w^(jk)
 *     inverse:  a_j = g^-j * n^-1 * sum_k A_k w^(-jk).
 * w = w_max^(2^(s - log_n)) where w_max = g0^((r-1)/2^s), g0 the field's
 * multiplicative generator (7 for BLS12-381 F_r, 5 for BN254 F_r, 22 for
 * BLS12-377 F_r) and s the 2-adicity of r - 1 (32, 28 and 47).
 *
 * Element layout (Section II: field elements as word-sized limbs): 8 x uint32
 * little-endian limbs = 32 bytes, Montgomery form X = x * 2^256 mod r,
 * canonical (0 <= X < r).  A vector is n such elements, contiguous, natural
 * order, 32-byte aligned.  Outputs are canonical Montgomery form too.
 *
 * Pointers named d_* are CUDA device pointers owned by the caller.  `stream`
 * is a cudaStream_t passed as void* (NULL = legacy default stream).  Every
 * execute call is stream-ordered and asynchronous: it returns once the work is
 * enqueued.  Errors the host can see (bad arguments, launch failures) are
 * returned at once; a device-side timeout of the persistent batch kernel is
 * returned by zkntt_sync_status() on the stream the launch ran on (each stream
 * has its own error word).  Plans are immutable after creation: one plan may be
 * executed from several host threads and streams at once, but only while the
 * device it was created on is current: every execute entry point returns
 * ZKNTT_EINVAL, before enqueuing anything, when another device is current.
 * Stream-ordered scratch comes from a memory pool private to this library (one
 * per device; freed blocks stay in it for reuse); the device's default pool is
 * not touched.
 */
#ifndef ZKNTT_H
#define ZKNTT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The scalar fields F_r of BLS12-381 (the curve the paper evaluates, Section
 * II), BN254, and BLS12-377 (also named in Section II). */
typedef enum { ZKNTT_BLS12_381_FR = 0, ZKNTT_BN254_FR = 1, ZKNTT_BLS12_377_FR = 2 } zkntt_field;
typedef enum { ZKNTT_FORWARD = 0, ZKNTT_INVERSE = 1 } zkntt_dir;
typedef enum {
    ZKNTT_OK = 0,
    ZKNTT_EINVAL = 1,        /* bad argument: null/misaligned pointer, log_n out of range, ... */
    ZKNTT_ENOMEM = 2,        /* device allocation failed */
    ZKNTT_ECUDA = 3,         /* a CUDA runtime call failed; see zkntt_last_cuda_error */
    ZKNTT_ETIMEOUT = 4,      /* a bounded device-side wait gave up (batch dependency never met) */
    ZKNTT_EUNSUPPORTED = 5   /* valid request the library does not implement */
} zkntt_status;

typedef enum {
    ZKNTT_TWIDDLE_AUTO = 0,     /* planner / tuner decides */
    ZKNTT_TWIDDLE_PRECOMP = 1,  /* full inter-pass twiddle tables resident in HBM */
    ZKNTT_TWIDDLE_OTF = 2       /* small split-exponent tables, twiddles formed in registers */
} zkntt_twiddle_mode;

typedef struct zkntt_plan_s *zkntt_plan;

/* One transform of a batch: input and output device vectors of the plan's size. */
typedef struct {
    const void *d_in;
    void *d_out;
} zkntt_io;

/* Optional planner overrides (zero-initialise and set what you need). */
typedef struct {
    int twiddle_mode;      /* zkntt_twiddle_mode */
    int num_passes;        /* 0 = planner's choice; else 1..4 */
    int digit_bits[4];     /* log2 sub-transform size per pass, top digit first; sum = log_n */
    int cols_per_cta[4];   /* columns per thread block per pass (1,2,4,8); 0 = planner's choice */
    int use_tuner;         /* 0 or 1: use a tuned schedule when one is known for this GPU
                              (zkntt_tuned.jsonl beside the library, then ZKNTT_TUNE_CACHE);
                              -1: never (planner heuristic only) */
    int ilp;               /* kernel variant: 1 = one butterfly per thread per stage step (3 blocks
                              per SM), 2 = two interleaved butterflies (2 blocks), 3 = one
                              butterfly with registers for 4 blocks, 4 = software-pipelined
                              stage loop (2 blocks), 5 = as 3 with twice the threads per
                              tile (for small transforms), 6 = as 3 with two tile
                              buffers (the next tile's loads overlap this tile's
                              arithmetic), 7 = as 1 with the stages of pair distance
                              16, 8 and 4 exchanged by warp shuffles instead of shared
                              memory; 0 = auto; outside 0..7 -> ZKNTT_EINVAL */
} zkntt_plan_options;

/*
 * Create a plan for one transform size/direction on the current CUDA device
 * (the transform of Section II-B; the coset form of Fig. 2).
 *   out          receives the plan handle (not written on failure)
 *   field        ZKNTT_BLS12_381_FR, ZKNTT_BN254_FR or ZKNTT_BLS12_377_FR
 *   log_n        1 .. the field's 2-adicity (32, 28 and 47); above 32 the
 *                vector and its scratch (2 x 2^log_n x 32 bytes, 512 GiB at
 *                2^33) exceed any device's memory: ZKNTT_ENOMEM
 *   dir          ZKNTT_FORWARD or ZKNTT_INVERSE
 *   coset_shift  NULL for a plain transform, else the shift g as 8 uint32
 *                Montgomery-form limbs (host memory, read during the call);
 *                must be nonzero and canonical.
 * The plan owns its device twiddle tables (allocated and filled here, freed by
 * zkntt_plan_destroy).  Without a tuned schedule or an explicit mode, the
 * inter-pass twiddles are precomputed tables (n entries for the first pass)
 * when those fit beside three vectors in the device memory free at creation,
 * else formed on the fly from split-exponent tables of about 2 sqrt(n)
 * entries.  Returns EINVAL on bad arguments, ENOMEM when the tables do not
 * fit, ECUDA on other CUDA failures.
 */
zkntt_status zkntt_plan_create(zkntt_plan *out, zkntt_field field, int log_n, zkntt_dir dir,
                               const uint32_t *coset_shift);

/* As zkntt_plan_create, with planner overrides (opts may be NULL): the schedule
 * parameters the paper asks to tune at run time (Section V-A). */
zkntt_status zkntt_plan_create_ex(zkntt_plan *out, zkntt_field field, int log_n, zkntt_dir dir,
                                  const uint32_t *coset_shift, const zkntt_plan_options *opts);

/* Free the plan's device tables (resource management; the paper has no
 * counterpart).  The caller must ensure no work using the plan is still in
 * flight.  NULL is accepted. */
zkntt_status zkntt_plan_destroy(zkntt_plan plan);

/* Size in bytes of the scratch vector an execution of this plan needs
 * (0 for single-pass sizes, else n * 32).  No counterpart in the paper. */
zkntt_status zkntt_plan_scratch_bytes(zkntt_plan plan, size_t *bytes);

/* Describe the plan: number of passes, digit bits per pass, twiddle mode and
 * the bytes of device tables it holds (any pointer may be NULL).  No
 * counterpart in the paper. */
zkntt_status zkntt_plan_describe(zkntt_plan plan, int *num_passes, int digit_bits[4],
                                 int *twiddle_mode, size_t *table_bytes);

/*
 * Run one transform: d_out = T(d_in), n = 2^log_n elements each (Section
 * II-B: A_k = sum_j a_j w^(jk); inverse and coset as described above).
 * d_in == d_out (in place) is allowed; partial overlap is EINVAL; a plan of
 * another device than the current one is EINVAL.  Scratch for multi-pass
 * sizes comes from the library's stream-ordered pool (allocated on `stream`,
 * released on `stream`).  The passes are enqueued on `stream` in order: the
 * first after all earlier work on it; the later ones as programmatic
 * dependents of the pass before (each waits for that pass's completion before
 * touching memory).  Work the caller enqueues afterwards sees the whole result
 * unless it is itself a programmatic dependent launch, which must then wait
 * (griddepcontrol.wait) before reading d_out.
 */
zkntt_status zkntt_execute(zkntt_plan plan, const void *d_in, void *d_out, void *stream);

/* As zkntt_execute (Section II-B) with caller-owned scratch (at least
 * zkntt_plan_scratch_bytes bytes, 32-byte aligned, not overlapping d_in/d_out);
 * allocates nothing. */
zkntt_status zkntt_execute_scratch(zkntt_plan plan, const void *d_in, void *d_out,
                                   void *d_scratch, size_t scratch_bytes, void *stream);

/*
 * End-to-end form for callers holding the data in HOST memory (the paper
 * attributes part of existing libraries' NTT time to host-device transfers,
 * Section IV-A; this form includes them): copies h_in
 * (n elements) to the device, runs the transform and copies the result to
 * h_out, all ordered on `stream` (device buffers come from the stream-ordered
 * pool and are released on the stream).  Returns once enqueued; h_out is valid
 * after the stream synchronises.  Pinned (page-locked) host buffers give
 * asynchronous copies; pageable ones are staged by the CUDA runtime.
 */
zkntt_status zkntt_execute_host(zkntt_plan plan, const void *h_in, void *h_out, void *stream);

/* As zkntt_execute_host with a caller-owned device work buffer instead of the
 * pool: d_work holds the vector and the plan's scratch, so work_bytes must be
 * at least n * 32 + zkntt_plan_scratch_bytes (32-byte aligned); nothing is
 * allocated in the call.  For callers that stream many transforms through
 * host memory (one work buffer per stream in flight). */
zkntt_status zkntt_execute_host_buffered(zkntt_plan plan, const void *h_in, void *h_out,
                                         void *d_work, size_t work_bytes, void *stream);

/* Largest scratch zkntt_execute_noalloc can use: 32 MiB, i.e. transforms of up
 * to 2^20 elements. */
#define ZKNTT_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

/*
 * zkntt_execute without any device allocation inside the call.  (The paper has
 * no counterpart; this exists for callers of this library.)  It is meant for
 * callers that must not allocate device memory while they run: for example a
 * host application that reserves the device's memory for itself up front and
 * does not let libraries call cudaMalloc, or a latency-critical loop that
 * cannot afford the device-wide synchronisation an allocation may cause.
 * The caller still passes the input and output vectors (and created the plan
 * beforehand); multi-pass sizes use a scratch array of
 * ZKNTT_NOALLOC_SCRATCH_BYTES that is a static device variable of this
 * library, so every GPU that loads the library holds those 32 MiB until the
 * process exits.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and keeps it; make that
 *     first call before any stream capture.
 *   - Plans whose scratch exceeds ZKNTT_NOALLOC_SCRATCH_BYTES (log_n > 20) are
 *     rejected with ZKNTT_EINVAL before anything is enqueued.
 *   - All calls on a device share the one array, which keeps whatever the last
 *     call left in it (the transform writes every scratch element before reading
 *     it, so nothing needs clearing).  Calls whose work can overlap on the GPU
 *     -- on different streams, or from several host threads -- race on the
 *     array; order them on one stream or synchronise between them.
 * Arguments, layout, aliasing and asynchrony as for zkntt_execute.
 */
zkntt_status zkntt_execute_noalloc(zkntt_plan plan, const void *d_in, void *d_out, void *stream);

/*
 * Run `count` independent transforms (each with its own plan; sizes, fields and
 * directions may differ) as ONE persistent kernel launch per field (the paper
 * finds provers issuing each transform as several short launches, Section
 * IV-A, and calls for batching and run-time tuning, Section V-A).  Work items (job,
 * pass, tile) are pulled from a device queue; a job's pass starts once all its
 * previous pass's tiles are done (bounded spin; on expiry the launch sets an
 * error word and returns, reported as ETIMEOUT).  ptrs[i] gives job i's
 * vectors.  In-place jobs are allowed; different jobs must not overlap.
 * Job scratch comes from the stream-ordered pool.
 */
zkntt_status zkntt_execute_batch(const zkntt_plan *plans, const zkntt_io *ptrs, int count,
                                 void *stream);

/*
 * As zkntt_execute_batch, for serving (transform sizes vary by application,
 * Section IV-A; the serving loop itself has no counterpart in the paper):
 * transforms are scheduled shortest
 * first, each one's passes back to back, and when transform i has completed on
 * the device the launch stores `epoch` into d_flags[i] with a system-scope
 * release, so a host thread polling host-mapped memory (zkntt_flags_create)
 * sees each result as soon as it is ready instead of at the end of the launch.
 * d_flags: count words of device-accessible memory; the caller picks a fresh
 * epoch per launch and may not reuse a slot before its flag is seen.
 */
zkntt_status zkntt_execute_batch_signal(const zkntt_plan *plans, const zkntt_io *ptrs, int count,
                                        uint32_t *d_flags, uint32_t epoch, void *stream);

/* Pinned host words that the device can write (zero-copy): host_view for
 * polling, device_view for zkntt_execute_batch_signal.  Zero-initialised.
 * Support for the serving form; no counterpart in the paper. */
zkntt_status zkntt_flags_create(int count, uint32_t **host_view, uint32_t **device_view);
zkntt_status zkntt_flags_destroy(uint32_t *host_view);

/*
 * Groth16 H polynomial (Fig. 2; Section IV-A counts seven transforms):
 *   a' = iNTT(a), b' = iNTT(b), c' = iNTT(c);
 *   A = cosetNTT_g(a'), B = cosetNTT_g(b'), C = cosetNTT_g(c');
 *   H_i = (A_i B_i - C_i) * (g^n - 1)^-1     (Z(x) = x^n - 1 on the coset g*w^i)
 *   d_h = cosetINTT_g(H)
 * with g the field's multiplicative generator.  d_a, d_b, d_c, d_h: n elements
 * each (inputs are read only; d_h must not overlap them).  d_scratch: 3 * n * 32
 * bytes of caller-owned device memory.  Runs the whole sequence as one
 * persistent launch (pointwise fused into the last transform's first pass);
 * further scratch comes from the library's stream-ordered pool.  log_n 1..28.
 */
zkntt_status zkntt_groth16_h(zkntt_field field, int log_n, const void *d_a, const void *d_b,
                             const void *d_c, void *d_h, void *d_scratch, void *stream);

/* As zkntt_groth16_h (Fig. 2), choosing the form: fused = 1 is the single
 * persistent launch; fused = 0 issues the seven transforms and the pointwise
 * kernel as separate launches (the form the paper finds in provers, Section
 * IV-A), for comparison. */
zkntt_status zkntt_groth16_h_ex(zkntt_field field, int log_n, const void *d_a, const void *d_b,
                                const void *d_c, void *d_h, void *d_scratch, int fused,
                                void *stream);

/*
 * The fused Groth16 H sequence (Fig. 2) captured once into a CUDA graph (the
 * launch-overhead reduction Section V-A points to): the capture
 * records the persistent launch and its stream-ordered scratch allocations
 * for these exact buffers; each zkntt_graph_launch replays it on `stream`
 * with no host-side work per transform.  `stream` must be a created stream
 * (not NULL) and idle during the call; the first call for a (field, log_n)
 * also builds the transform plans before capturing.  The buffers must stay
 * valid for the graph's lifetime.
 */
typedef struct zkntt_graph_s *zkntt_graph;

zkntt_status zkntt_groth16_graph_create(zkntt_graph *out, zkntt_field field, int log_n,
                                        const void *d_a, const void *d_b, const void *d_c, void *d_h,
                                        void *d_scratch, void *stream);
zkntt_status zkntt_graph_launch(zkntt_graph graph, void *stream);
zkntt_status zkntt_graph_destroy(zkntt_graph graph);

/* The library's stream-ordered scratch pool on the current device (memory
 * management; no counterpart in the paper): *reserved_bytes is the device
 * memory the pool holds, *used_bytes the part handed out to executions in
 * flight.  The difference is free for the library's next executions although
 * cudaMemGetInfo counts it as used; a caller admitting work by free device
 * memory (a serving loop) adds it back. */
zkntt_status zkntt_pool_info(size_t *reserved_bytes, size_t *used_bytes);

/* Static text for a status code (error reporting; no counterpart in the paper). */
const char *zkntt_status_str(zkntt_status status);

/* The last CUDA error code this library saw on the calling thread (0 = none).
 * Error reporting; no counterpart in the paper. */
zkntt_status zkntt_last_cuda_error(int *err);

/* Wait for `stream` and report any device-side error word (ETIMEOUT) or CUDA
 * error raised by work this library enqueued on it; the stream's error word is
 * cleared once reported.  Each stream has its own word (the first 1023 streams
 * that run a batch launch on a device; later ones share one more), so a
 * timeout on one stream is not reported on another.  A captured launch
 * (zkntt_groth16_graph_create) reports to the word of the stream it was
 * captured on.  Error reporting; no counterpart in the paper. */
zkntt_status zkntt_sync_status(void *stream);

/* Fault-injection self-test of the persistent kernel's bounded wait (failure
 * detection; no counterpart in the paper): launches
 * it with a single work item whose dependency can never be met (injected on
 * the host) and a device-side wait limit of timeout_ms, then returns what
 * zkntt_sync_status reports -- ZKNTT_ETIMEOUT when the bound works.  No GPU
 * fault is involved; the context stays usable. */
zkntt_status zkntt_selftest_timeout(int timeout_ms, void *stream);

/* The launch half of zkntt_selftest_timeout (failure detection; no counterpart
 * in the paper): enqueues the same never-satisfied single-item launch with a
 * wait limit of timeout_ms (1..10000, else ZKNTT_EINVAL) on `stream` and
 * returns once enqueued.  When the wait gives up, the launch sets `stream`'s
 * error word, so zkntt_sync_status(stream) returns ZKNTT_ETIMEOUT while the
 * other streams' words stay clear. */
zkntt_status zkntt_inject_timeout(int timeout_ms, void *stream);

/* Self-test of the plan-device check (argument validation; no counterpart in
 * the paper).  A plan's tables live on the device that was current when it was
 * created, and every execute entry point returns ZKNTT_EINVAL, before enqueuing
 * anything, when another device is current.  This creates a 16-element plan
 * on the current device, marks a copy of it as belonging to another device,
 * passes the copy to each of the execute entry points (zkntt_execute, _scratch,
 * _host, _host_buffered, _noalloc, _batch, _batch_signal) with real 16-element
 * buffers, and reports how many were called (*checked) and how many returned
 * ZKNTT_EINVAL (*rejected).  Synchronous; frees everything it created. */
zkntt_status zkntt_selftest_device_check(int *checked, int *rejected);

/* Field information (the prime fields of Section II; the generator is this
 * library's reading, the paper prints none): modulus and Montgomery form of the
 * generator, 8 limbs each (host memory, either may be NULL), and the
 * 2-adicity. */
zkntt_status zkntt_field_info(zkntt_field field, uint32_t modulus[8], uint32_t generator_mont[8],
                              int *two_adicity);

/* Elementwise field operations on device vectors of n elements (FF_mul,
 * FF_add and FF_sub of Section IV-B; test and calibration entry points for
 * the butterfly arithmetic):
 *   op 0: c = a * b (Montgomery product a b 2^-256 mod r, canonical; a must be
 *         canonical, b may be any 256-bit value)
 *   op 1: c = a + b mod r      op 2: c = a - b mod r
 *   op 3: c = a + r - b, the unreduced butterfly difference (in (0, 2r) for
 *         canonical a, b; it feeds the product as its second operand)
 * Inputs of ops 1-3 must be canonical.  op outside 0..3 -> ZKNTT_EINVAL.
 */
zkntt_status zkntt_field_op(zkntt_field field, int op, const void *d_a, const void *d_b, void *d_c,
                            size_t n, void *stream);

/* Scale by a geometric sequence: d_out[i] = d_x[i] * c * base^i for i < n
 * (c and base: 8 Montgomery limbs in host memory, canonical; in place
 * allowed).  This is the twiddle step of the four-step decomposition of the
 * transform (Section II-B: a block NTT is bounded by shared memory, so large
 * transforms are split into sub-transforms joined by twiddle factors), used
 * when the sub-transforms run on different GPUs; with base = 1 it multiplies
 * by the constant c.  Tables of about 2 sqrt(n) powers come from the
 * library's stream-ordered pool for the call.  Non-canonical c or base,
 * null or misaligned pointers, partial overlap -> ZKNTT_EINVAL. */
zkntt_status zkntt_scale_powers(zkntt_field field, const void *d_x, void *d_out, size_t n,
                                const uint32_t *c_mont, const uint32_t *base_mont, void *stream);

/* G-point transforms over whole blocks (G = 2^log_g, log_g 1..3): with the
 * input laid out as G blocks of b elements (element r * b + i), for every
 * column i < b
 *     d_out[k * b + i] = sum_r d_in[r * b + i] * w^(r k)      (r, k < G)
 * where w is the field's root of order G (its inverse when inverse != 0; no
 * 1/G factor).  This is the last step of the four-step decomposition
 * (Section II-B) when the sub-transforms of the other digit live on
 * different GPUs: the sharded transform applies it to the blocks it receives
 * from the G ranks.  In place allowed; partial overlap, bad pointers or
 * log_g outside 1..3 -> ZKNTT_EINVAL.  Allocates nothing. */
zkntt_status zkntt_block_dft(zkntt_field field, int log_g, size_t b, const void *d_in, void *d_out,
                             int inverse, void *stream);

/* Groth16 pointwise step on its own (the (A B - C) / Z step of Fig. 2):
 * d_h_i = (a_i b_i - c_i) * z, z given as 8 Montgomery limbs in host memory. */
zkntt_status zkntt_pointwise(zkntt_field field, const void *d_a, const void *d_b, const void *d_c,
                             const uint32_t *z_mont, void *d_h, size_t n, void *stream);

/* Result of zkntt_tune: the fastest schedule found. */
typedef struct {
    int num_passes;
    int digit_bits[4];
    int cols_per_cta[4];
    int twiddle_mode;
    int ilp;
    float ms;            /* median time of one transform with that schedule */
} zkntt_tune_result;

/*
 * Autotuner (the paper's call for runtime parameter tuning, Section V-A): time
 * up to `max_candidates` schedules (pass split, columns per block, twiddle
 * mode) for one plain transform of 2^log_n elements on the current device with
 * CUDA events, remember the fastest for this GPU (and append it to the file
 * named by ZKNTT_TUNE_CACHE, one JSON object per line) and return it in *best
 * (may be NULL).  Plans created afterwards use it (unless opts->use_tuner < 0
 * or the caller forces a digit split).  Schedules tuned ahead of time ship in
 * zkntt_tuned.jsonl beside the library.  Uses
 * 3 * n * 32 bytes of temporary device memory; synchronous.
 */
zkntt_status zkntt_tune(zkntt_field field, int log_n, zkntt_dir dir, int max_candidates,
                        zkntt_tune_result *best);

/*
 * Integer-pipe calibration (Sections IV-B and IV-C find FF_mul bound by the
 * 32-bit integer pipe): runs `iters` Montgomery products per thread on a
 * grid of `blocks` x `threads` (register-resident, no memory traffic inside
 * the loop) and writes one checksum word per thread to d_sink.  Used to
 * measure the sustained 32-bit multiply-add rate that bounds the transform.
 */
zkntt_status zkntt_mulbench(zkntt_field field, int blocks, int threads, int iters, void *d_sink,
                            void *stream);

/*
 * Peak calibration of the 32-bit integer multiply-add (IMAD) rate, the
 * denominator of the transform's roofline (Sections IV-B and IV-C find FF_mul
 * bound by the INT32 pipe and weight IMAD in its integer roofline), and of the
 * multiply forms a Montgomery product is built from: a grid of `blocks` x
 * `threads` (32..1024) runs `iters` steps of eight independent
 * register-resident chains per thread and writes one checksum word per thread
 * to d_sink.  One step is, by mode:
 *   0  mad.lo.u32     (one 32-bit multiply-add: the peak rate)
 *   1  mad.wide.u32   (32 x 32 -> 64 multiply with a 64-bit addend)
 *   2  mul.wide.u32   (32 x 32 -> 64 multiply, no addend)
 *   3  mad.hi.u32     (high half of a 32 x 32 product plus an addend)
 *   4  mad.lo.cc.u32 + madc.hi.u32 (a carry-chained pair: two instructions)
 * 8 * iters steps per thread; time it with CUDA events on `stream`.  mode
 * outside 0..4 or bad sizes -> ZKNTT_EINVAL.
 */
zkntt_status zkntt_imadbench(int mode, int blocks, int threads, int iters, void *d_sink,
                             void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ZKNTT_H */
