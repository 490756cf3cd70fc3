/*
 * prand.h -- C ABI of a GB300 (sm_103a) library that generates many independent
 * streams of uniform pseudorandom numbers with the eleven generators of PRAND
 * (Barash & Shchur, "PRAND: GPU accelerated parallel random number generation
 * library", Comput. Phys. Commun. 185 (2014) 1343).
 *
 * The problem statement follows the paper: "fill an array in GPU memory with
 * the next `length` numbers of a generator state" (Sec. 6; Sec. 7.5,
 * rng_generate_gpu_array_, _float_, _double_) and "initialise stream number k
 * by block splitting" (Sec. 5; Sec. 7.1, rng_init_sequence_; Table 4), here for
 * n streams at once.
 *
 * Conventions for every entry point:
 *   - Pointers named dev_* are CUDA device pointers owned by the caller; host_*
 *     are host pointers owned by the caller.  The library never frees them.
 *   - A prand_stream_t is a cudaStream_t (NULL = the legacy default stream).
 *   - Every call returns a prand_status_t.  Nothing aborts, nothing traps on
 *     the device; a CUDA error is reported as PRAND_ERR_CUDA.
 *   - Generation calls are asynchronous on the given stream; state creation,
 *     stream initialisation, skip-ahead and state get/set complete before they
 *     return.
 *   - A handle is bound to the CUDA device that was current at prand_create;
 *     every later call on it must be made with that device current.
 *   - Calls on the same handle must not overlap (no internal locking per
 *     handle).  Different handles are independent.
 */
#ifndef PRAND_H
#define PRAND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct prand_handle_s *prand_handle_t;
typedef void *prand_stream_t; /* a cudaStream_t */

/* The eleven generators (Table 2).  The order is part of the ABI. */
typedef enum {
    PRAND_MT19937 = 0,  /* Matsumoto-Nishimura 1998; Sec. 5.4                       */
    PRAND_MRG32K3A = 1, /* L'Ecuyer 1999; Sec. 5.2                                  */
    PRAND_LFSR113 = 2,  /* L'Ecuyer 1999, four Tausworthe components; Sec. 5.3      */
    PRAND_GM19 = 3,     /* torus-map ensembles, eq. (rec1) with Table 2's (k,q,g,v) */
    PRAND_GM29 = 4,
    PRAND_GM31 = 5,
    PRAND_GM55 = 6,
    PRAND_GM61 = 7,
    PRAND_GQ58_1 = 8,
    PRAND_GQ58_3 = 9,
    PRAND_GQ58_4 = 10,
    PRAND_NUM_GENERATORS = 11
} prand_gen_t;

typedef enum {
    PRAND_OK = 0,
    PRAND_ERR_ARG = 1,             /* null handle/pointer, bad enum, size overflow        */
    PRAND_ERR_ALIGN = 2,           /* dev_out not aligned to its element size             */
    PRAND_ERR_NOMEM = 3,           /* device or host allocation failed                    */
    PRAND_ERR_CUDA = 4,            /* a CUDA runtime call or kernel launch failed         */
    PRAND_ERR_STATE = 5,           /* call out of order (e.g. generate before init) or a
                                      state blob of the wrong generator/size/version      */
    PRAND_ERR_TIMEOUT = 6,         /* a bounded device wait gave up                       */
    PRAND_WARN_STREAM_OVERLAP = 7  /* success, but first_stream + n_streams exceeds the
                                      Table 4 capacity of the generator, so streams may
                                      overlap within the generator's period             */
} prand_status_t;

/* Seed value meaning "the paper's default initial state" (rng_init_, Sec. 7.1):
 * MT19937 init_genrand(5489); MRG32K3A all six words 12345; LFSR113 all four
 * words 987654321; GM/GQ base pair (1, 1). */
#define PRAND_SEED_DEFAULT UINT64_MAX

/* Element types of prand_request_t.dtype. */
#define PRAND_DTYPE_U32 0
#define PRAND_DTYPE_F32 1
#define PRAND_DTYPE_F64 2

/* Create a handle for generator `gen` and build its base state on the current
 * device (rng_init_, Sec. 7.1).  seed == PRAND_SEED_DEFAULT gives the default
 * state; MT19937 seeds below 2^32 use init_genrand(seed), wider seeds
 * init_by_array({lo32, hi32}); the other generators expand the seed with
 * SplitMix64.  The first handle of a generator family on a device also builds
 * that family's device jump tables (MT19937: the polynomials x^(2^b) mod phi,
 * b < 512, Sec. 5.4).  On success *h owns its device memory until
 * prand_destroy.  Errors: PRAND_ERR_ARG (h NULL, gen out of range),
 * PRAND_ERR_NOMEM, PRAND_ERR_CUDA. */
prand_status_t prand_create(prand_handle_t *h, prand_gen_t gen, uint64_t seed);

/* Allocate and initialise n_streams block-split streams: stream j of the handle
 * is stream (first_stream + j) of the generator, i.e. the base state advanced
 * by (first_stream + j) * L (Sec. 5; Table 4: the init_sequence variant with
 * the most sequences: L = 6e6 GM19; 8e7 GM29, GM31, GQ58.x; 1e10 GM55, GM61;
 * 2^34 LFSR113; 2^127 MRG32K3A; 2^432 MT19937).  The jump is exact for any
 * 64-bit first_stream.  Replaces streams set up by an earlier call.
 * Returns PRAND_WARN_STREAM_OVERLAP (after doing the work) when
 * first_stream + n_streams exceeds the Table 4 number of sequences.
 * Errors: PRAND_ERR_ARG (n_streams == 0 or first_stream + n_streams overflows),
 * PRAND_ERR_NOMEM, PRAND_ERR_CUDA. */
prand_status_t prand_init_streams(prand_handle_t h, uint64_t first_stream, uint64_t n_streams);

/* The same with a stream-initialisation variant of Table 4:
 * PRAND_VARIANT_DEFAULT (init_sequence / init_short_sequence, the one
 * prand_init_streams uses), PRAND_VARIANT_MEDIUM (init_medium_sequence) or
 * PRAND_VARIANT_LONG (init_long_sequence).  A variant trades the number of
 * streams for their length: stream k starts k * L_v outputs after the base,
 * with (N_max, L_v) the variant's row of Table 4 (block length: the printed
 * maximal length for GM/GQ, 2^80 for LFSR113 long); for GM/GQ the base
 * ensemble's points are spaced N_max L_v apart, so each variant has its own
 * base.  Medium exists for GM29, GM31 and GQ58.x; long for those and GM55,
 * GM61, LFSR113; MRG32K3A and MT19937 have the default only.
 * Errors: as prand_init_streams, and PRAND_ERR_ARG for a variant Table 4 does
 * not list for the generator. */
#define PRAND_VARIANT_DEFAULT 0
#define PRAND_VARIANT_MEDIUM 1
#define PRAND_VARIANT_LONG 2
prand_status_t prand_init_streams_variant(prand_handle_t h, int32_t variant, uint64_t first_stream,
                                          uint64_t n_streams);

/* Streams spaced 2^log2_spacing outputs apart: stream k = the base advanced by
 * k * 2^log2_spacing (for GM/GQ the default variant's base ensemble).  This is
 * the layout of the paper's skip-ahead study (Sec. 4, Table 3): output 0 of
 * streams 0, 1, 2, ... is the subsequence that skips 2^n values at each step,
 * and output i of them is the same subsequence started i values later.
 * log2_spacing <= 448 for MT19937 and <= 127 for the other generators.  No
 * capacity warning: streams overlap once more than 2^log2_spacing outputs are
 * drawn from one, which the caller controls.  Generation, skip-ahead and
 * checkpoints work as after prand_init_streams.
 * Errors: as prand_init_streams, and PRAND_ERR_ARG for a spacing out of range. */
prand_status_t prand_init_streams_spaced(prand_handle_t h, uint32_t log2_spacing, uint64_t first_stream,
                                         uint64_t n_streams);

/* Write the next n_per_stream outputs of every stream, stream-major:
 * dev_out[j * n_per_stream + i] = output i of stream j (rng_generate_gpu_array_,
 * Sec. 6).  Each stream continues where the previous generate call on the
 * handle stopped; the u32, f32 and f64 calls share that position.
 * u32: the generator's 32-bit output (MRG32K3A: z in [1, m1]).
 * f32: (u >> 8) * 2^-24 in [0, 1).
 * f64: u * 2^-32 in [0, 1); MRG32K3A: z * RN(1 / (m1 + 1)) in (0, 1).
 * dev_out must hold n_streams * n_per_stream elements and be aligned to its
 * element size (16-byte alignment enables vector stores).  Any n_per_stream
 * >= 0 is accepted (0 is a no-op).  Asynchronous on `stream`.
 * Errors: PRAND_ERR_ARG, PRAND_ERR_ALIGN, PRAND_ERR_STATE (no streams yet),
 * PRAND_ERR_CUDA. */
prand_status_t prand_generate_u32(prand_handle_t h, uint32_t *dev_out, uint64_t n_per_stream, prand_stream_t stream);
prand_status_t prand_generate_f32(prand_handle_t h, float *dev_out, uint64_t n_per_stream, prand_stream_t stream);
prand_status_t prand_generate_f64(prand_handle_t h, double *dev_out, uint64_t n_per_stream, prand_stream_t stream);

/* The same fills into HOST memory (the paper's host-array fill,
 * rng_generate_array_, Sec. 7.5): host_out[j * n_per_stream + i] = output i of
 * stream j, the values prand_generate_* would write.  host_out is
 * caller-owned host memory aligned to the element size.  Page-locked memory
 * (cudaMallocHost / cudaHostAlloc / cudaHostRegister, mapped into the device's
 * address space as every page-locked allocation is under unified addressing)
 * is written by the generation kernels directly, over the host link, with no
 * staging.  Pageable memory works too: its outputs are generated on the device
 * in blocks that fit a staging area owned by the handle (two buffers of 256
 * MiB, or PRAND_HOST_STAGE_BYTES from the environment at the handle's first
 * pageable host fill, allocated then and freed by prand_destroy), each block's
 * copy overlapping the next block's generation.  Generation runs on `stream`
 * (after work already queued there); the call returns once every output is in
 * host_out.
 * Errors: PRAND_ERR_ARG, PRAND_ERR_ALIGN, PRAND_ERR_STATE, PRAND_ERR_NOMEM
 * (staging), PRAND_ERR_CUDA. */
prand_status_t prand_generate_host_u32(prand_handle_t h, uint32_t *host_out, uint64_t n_per_stream, prand_stream_t stream);
prand_status_t prand_generate_host_f32(prand_handle_t h, float *host_out, uint64_t n_per_stream, prand_stream_t stream);
prand_status_t prand_generate_host_f64(prand_handle_t h, double *host_out, uint64_t n_per_stream, prand_stream_t stream);

/* The streams as single-stream states for user code (prand_device.h, the
 * paper's single-threaded interface, Sec. 7.3): prand_export_states writes
 * one struct per stream, stream j at index j (prand_mt19937_state,
 * prand_mrg32k3a_state, prand_lfsr113_state or prand_gm_state, of
 * prand_device_state_bytes(gen) bytes each), at the streams' current
 * positions; prand_import_states reads them back, so the handle continues from
 * wherever user code left each stream.  dev_states: caller-owned device memory
 * of n_streams structs, 8-byte aligned for GM/GQ and 4-byte aligned otherwise.
 * MT19937 handles keep one in-block index for all streams: an import whose
 * structs disagree on it returns PRAND_ERR_STATE and changes nothing (this
 * check waits for `stream`).  The output position of prand_query is not
 * changed by an import.  Asynchronous on `stream` otherwise.
 * prand_device_state_bytes returns 0 for an unknown generator.
 * Errors: PRAND_ERR_ARG, PRAND_ERR_ALIGN, PRAND_ERR_STATE, PRAND_ERR_NOMEM,
 * PRAND_ERR_CUDA. */
uint64_t prand_device_state_bytes(prand_gen_t gen);
prand_status_t prand_export_states(prand_handle_t h, void *dev_states, prand_stream_t stream);
prand_status_t prand_import_states(prand_handle_t h, const void *dev_states, prand_stream_t stream);

/* The MT19937 jump polynomial g(x) = x^(2^b) mod phi(x), b = 0..511 (Sec. 5.4:
 * the stored family g_v with v = 2^b; phi is the characteristic polynomial of
 * the one-output state transition A, degree 19937).  A state advanced by 2^b
 * outputs is g(A) applied to it (eq. (g_v)), which a kernel of the caller's can
 * evaluate on states from prand_export_states.  Writes 624 words to host_out
 * (caller-owned host memory): the coefficient of x^i is bit i % 32 of word
 * i / 32; bits 19937..19967 are zero.  Host-only and thread-safe; the first
 * call of the process computes the family (phi by Berlekamp-Massey, then 511
 * squarings mod phi, about 0.1 s), later calls copy.
 * Errors: PRAND_ERR_ARG (b > 511 or host_out NULL), PRAND_ERR_STATE (the
 * family could not be computed; not expected). */
prand_status_t prand_mt_jump_polynomial(uint32_t b, uint32_t *host_out);

/* Advance every stream of the handle by the 256-bit offset offset_le[0] +
 * 2^64 offset_le[1] + 2^128 offset_le[2] + 2^192 offset_le[3] outputs
 * (rng_skipahead_, Sec. 7.2; jump methods of Sec. 5.1-5.4).
 * Errors: PRAND_ERR_ARG, PRAND_ERR_STATE (no streams), PRAND_ERR_CUDA. */
prand_status_t prand_skipahead(prand_handle_t h, const uint64_t offset_le[4]);

/* Advance every stream by a * 2^b outputs (the paper's MT19937 skip-ahead
 * form, N = a 2^b < 2^512, Sec. 7.9); for MT19937 a 2^b may reach 2^512, for
 * the other generators it must stay below 2^256 (it is then prand_skipahead
 * with that offset).  a = 0 is a no-op.  Returns after the work completes.
 * Errors: PRAND_ERR_ARG (out of range), PRAND_ERR_STATE, PRAND_ERR_CUDA. */
prand_status_t prand_skipahead_pow2(prand_handle_t h, uint64_t a, uint32_t b);

/* Copy the full state of all streams into a host buffer (checkpoint), as a
 * versioned blob that prand_set_state accepts on a handle of the same
 * generator (the paper's state copy between host and device, Sec. 7).
 * If host_buf is NULL, only *bytes is set to the size needed.
 * Errors: PRAND_ERR_ARG (bytes NULL or *bytes too small), PRAND_ERR_STATE,
 * PRAND_ERR_CUDA. */
prand_status_t prand_get_state(prand_handle_t h, void *host_buf, size_t *bytes);
prand_status_t prand_set_state(prand_handle_t h, const void *host_buf, size_t bytes);

/* Number of streams of the handle and the per-stream output position
 * (outputs produced since prand_init_streams, modulo 2^64).
 * Errors: PRAND_ERR_ARG. */
prand_status_t prand_query(prand_handle_t h, uint64_t *first_stream, uint64_t *n_streams, uint64_t *position);

/* Free the handle's device memory (the handle's counterpart of the paper's
 * state struct, Sec. 7.1, going out of scope).  h == NULL is a no-op; returns
 * PRAND_OK. */
prand_status_t prand_destroy(prand_handle_t h);

/* A static English string for a status code. */
const char *prand_status_string(prand_status_t status);

/* Number of device kernels this library has launched in the process (no
 * counterpart in the paper; a launch count for benchmarks).  Cannot fail. */
uint64_t prand_kernel_launches(void);

/* The float maps on their own (Sec. 7.3 asks only for outputs uniform in
 * [0, 1); the exact maps are this library's reading, the same ones every
 * prand_generate_f32 / _f64 call applies):
 *   map = PRAND_DTYPE_F32:   out[i] = (float)(in[i] >> 8) * 2^-24     in [0, 1)
 *   map = PRAND_DTYPE_F64:   out[i] = (double)in[i] * 2^-32           in [0, 1), exact
 *   map = PRAND_MAP_MRG_F64: out[i] = (double)in[i] * RN(1 / (m1 + 1)), one
 *                            round-to-nearest multiply (MRG32K3A's map; in (0, 1)
 *                            for its outputs z in [1, m1])
 * dev_in: n caller-owned 32-bit words in device memory (4-byte aligned);
 * dev_out: n floats or doubles, caller-owned, aligned to the element size (may
 * not overlap dev_in).  Asynchronous on `stream`.
 * Errors: PRAND_ERR_ARG (null pointer with n > 0, unknown map), PRAND_ERR_ALIGN,
 * PRAND_ERR_CUDA (launch failure). */
#define PRAND_MAP_MRG_F64 3
prand_status_t prand_convert(const uint32_t *dev_in, uint64_t n, int32_t map, void *dev_out, prand_stream_t stream);

/* ---- Batched requests (no counterpart in the paper: many streams of mixed
 * generators in one launch; each request is the paper's block-split stream,
 * Sec. 5 / Table 4, filled as in Sec. 6) ----
 * One batched request: `length` outputs of stream `stream` of generator `gen`
 * (seeded with the batch's seed), starting at the stream's beginning, written
 * to dev_out (caller-owned, aligned to the element size of `dtype`). */
typedef struct {
    int32_t gen;      /* prand_gen_t */
    int32_t dtype;    /* PRAND_DTYPE_U32 / _F32 / _F64 */
    uint64_t stream;  /* any 64-bit stream index (block splitting, Table 4) */
    uint64_t length;  /* outputs to write */
    void *dev_out;    /* device pointer */
} prand_request_t;

/* Run n requests of mixed generators and uneven lengths in one persistent
 * launch (asynchronous on `stream`): each request's jump to its stream and to
 * the start of each of its sections (block splitting, Sec. 5 / Table 4) is
 * fused in front of its generation; warps take tiles (sections of requests)
 * from a shared counter, longest first.  Each request's output equals
 * prand_init_streams(stream, 1) then prand_generate_<dtype>(length) on a handle
 * created with the same seed.  The request array may be reused as soon as the
 * call returns; the library keeps its own copy of the work list.
 * Errors: PRAND_ERR_ARG, PRAND_ERR_ALIGN, PRAND_ERR_NOMEM, PRAND_ERR_CUDA. */
prand_status_t prand_batch_run(const prand_request_t *reqs, size_t n, uint64_t seed, prand_stream_t stream);

/* The same requests, one ordinary stream-initialisation launch and one
 * generation launch per request (no fusion, no persistent scheduling); the
 * comparison point for prand_batch_run.  Each stream is reached by the same
 * jump method the batched launch uses (for MT19937, one window polynomial per
 * nonzero byte of the stream index), so the two differ only in how the
 * work is launched.  Returns after the work completes.
 * Errors: as prand_batch_run. */
prand_status_t prand_batch_run_per_request(const prand_request_t *reqs, size_t n, uint64_t seed,
                                           prand_stream_t stream);

/* A prepared batch: the work list is planned and uploaded once and the launch
 * is captured in a CUDA graph, so prand_batch_plan_launch replays it with one
 * graph launch.  Outputs go to the requests' dev_out pointers on every launch.
 * Errors: PRAND_ERR_ARG, PRAND_ERR_ALIGN, PRAND_ERR_NOMEM, PRAND_ERR_CUDA;
 * launch: PRAND_ERR_STATE if another device is current. */
typedef struct prand_batch_plan_s *prand_batch_plan_t;
prand_status_t prand_batch_plan_create(prand_batch_plan_t *plan, const prand_request_t *reqs, size_t n, uint64_t seed);
prand_status_t prand_batch_plan_launch(prand_batch_plan_t plan, prand_stream_t stream);
prand_status_t prand_batch_plan_destroy(prand_batch_plan_t plan);

/* Tile tuner (no counterpart in the paper): times the batch (as a graph
 * plan, mean of three launches) over the launch parameters and keeps the
 * fastest for later batches on this device: first the two section lengths
 * (outputs per lane of the thread-per-section tiles -- MRG32K3A, LFSR113 and
 * the thread-per-stream GM/GQ ensembles -- and outputs per warp of the
 * lane-per-point GM/GQ tiles: 2048, 8192 or 32768 each), then, at the best
 * lengths, the threads per block (64 or 128) and the staged row size (128 or
 * 256 bytes, i.e. 32 or 64 u32 outputs per row store) of the kernel build
 * that runs MRG32K3A, LFSR113 and the lane-per-point GM/GQ tiles.  Reports the
 * choice (any output pointer may be NULL).  If the environment variable
 * PRAND_TUNE_CACHE names a file, the result is written there and read back by
 * later processes.  The requests' outputs are written (several times).
 * Errors: as prand_batch_run. */
prand_status_t prand_batch_autotune(const prand_request_t *reqs, size_t n, uint64_t seed, prand_stream_t stream,
                                    uint32_t *seclen_mrg_lfsr, uint32_t *seclen_gm, uint32_t *block,
                                    uint32_t *row_bytes, float *best_ms);

/* Sets the batched launch parameters the tuner chooses (same meanings and
 * allowed values: section lengths multiples of 4, block 64 or 128, row_bytes
 * 128 or 256) for later batches and plans on the current device, e.g. from a
 * configuration kept elsewhere.  Errors: PRAND_ERR_ARG, PRAND_ERR_CUDA. */
prand_status_t prand_batch_set_params(uint32_t seclen_mrg_lfsr, uint32_t seclen_gm, uint32_t block,
                                      uint32_t row_bytes);

/* ---- Request server (no counterpart in the paper: continuous batching of
 * stream requests, with stream states resident on the device) ----
 * A request (generator, stream index, length, element type) returns the next
 * `length` outputs of that stream: the server keeps each stream it has served
 * resident on the device and continues it on the next request; a stream seen
 * for the first time starts from the seed's base advanced by k * L (Table 4).
 * A worker thread admits pending requests in arrival order while the output
 * arena has room, launches them as batches of the persistent kernel on
 * several CUDA streams (batches overlap on the device), and keeps requests on
 * the same stream in order.  When a generator's slots are all taken, the least
 * recently used idle stream's state moves to host memory and is restored on
 * its next request, so results never depend on the order of other streams. */
typedef struct prand_server_s *prand_server_t;
typedef struct {
    uint64_t completed, samples;  /* requests finished, outputs produced            */
    uint64_t hits, misses;        /* requests that continued a resident stream / not */
    uint64_t spills, restores;    /* states moved to host memory and back           */
    uint64_t batches, pending;    /* batches launched, requests waiting now         */
    uint64_t tiles;               /* work tiles launched                            */
    double worker_busy_s;         /* worker time spent planning and launching       */
    uint64_t arena_used_bytes;    /* output bytes held now                          */
    uint64_t arena_free_blocks;   /* free fragments of the output arena now         */
    uint64_t arena_top_bytes;     /* highest output offset handed out so far        */
    uint64_t flights_busy;        /* batches on the device now                      */
    double gpu_busy_s;            /* summed device time of the finished batches     */
} prand_server_stats_t;

/* output_bytes: device arena for outputs (a request whose output does not fit
 * is refused at submit); slots_per_generator: resident streams per generator.
 * The server is bound to the current device; its worker thread makes that
 * device current itself.  It keeps up to 32 batches in flight, each on its own
 * stream; the process should set CUDA_DEVICE_MAX_CONNECTIONS=32 (the driver
 * default is 8) before CUDA starts, or flights that share a hardware queue wait
 * behind one another's long batches.  Errors: PRAND_ERR_ARG, PRAND_ERR_NOMEM,
 * PRAND_ERR_CUDA. */
prand_status_t prand_server_create(prand_server_t *srv, uint64_t seed, uint64_t output_bytes,
                                   uint32_t slots_per_generator);
/* Queue a request; *id identifies it.  Thread-safe.  Errors: PRAND_ERR_ARG. */
prand_status_t prand_server_submit(prand_server_t srv, int32_t gen, uint64_t stream, uint64_t length, int32_t dtype,
                                   uint64_t *id);
/* *done = 1 once the outputs are on the device at *dev_out (valid until
 * prand_server_release); *latency_s = completion time - submit time.
 * Errors: PRAND_ERR_ARG (null server, unknown id). */
prand_status_t prand_server_query(prand_server_t srv, uint64_t id, int32_t *done, void **dev_out, double *latency_s);
/* Copy the first `bytes` of a completed request's output to host memory
 * (synchronous).  Errors: PRAND_ERR_ARG (null pointer, more bytes than the
 * output), PRAND_ERR_STATE (unknown or unfinished id), PRAND_ERR_CUDA. */
prand_status_t prand_server_read(prand_server_t srv, uint64_t id, void *host_dst, uint64_t bytes);
/* Ids of requests completed since the last call (at most cap; *n = count).
 * Errors: PRAND_ERR_ARG (null server or n, ids NULL with cap > 0). */
prand_status_t prand_server_completed(prand_server_t srv, uint64_t *ids, size_t cap, size_t *n);
/* Return a completed request's output memory to the arena.
 * Errors: PRAND_ERR_ARG (null server), PRAND_ERR_STATE (unknown or unfinished id). */
prand_status_t prand_server_release(prand_server_t srv, uint64_t id);
/* Counters of the server so far.  Errors: PRAND_ERR_ARG (null pointer). */
prand_status_t prand_server_stats(prand_server_t srv, prand_server_stats_t *stats);
/* Stops the worker after the batches in flight; outstanding outputs are freed.
 * srv == NULL is a no-op. */
prand_status_t prand_server_destroy(prand_server_t srv);
/* Open-loop load driver: submits reqs[i] (dev_out ignored) arrival_s[i] seconds
 * after the call (arrival_s ascending), releases outputs as they complete, and
 * writes each request's latency; *wall_s = time until the last completion.
 * Errors: PRAND_ERR_ARG (null arrays with n > 0, a request submit refuses). */
prand_status_t prand_server_replay(prand_server_t srv, const prand_request_t *reqs, const double *arrival_s, size_t n,
                                   double *latency_s, double *wall_s);

/* Statistical tests of generated words (the paper tests the generators and
 * their skip-ahead subsequences with TestU01, Secs. 3-4, Tables 1 and 3; these are
 * three classical tests from Knuth, TAOCP vol. 2, Sec. 3.3.2):
 *   PRAND_TEST_FREQUENCY  the top `bits` bits of each word select one of
 *                         2^bits cells (1 <= bits <= 12);
 *   PRAND_TEST_SERIAL     non-overlapping pairs (u[2i], u[2i+1]), i < n/2; the
 *                         cell is (top bits of u[2i]) * 2^bits + (top bits of
 *                         u[2i+1]) (1 <= bits <= 6, 4^bits cells; an odd last
 *                         word is not used);
 *   PRAND_TEST_GAP        u is a hit when lo <= u < hi (lo < hi <= 2^32); each
 *                         hit closes a gap of r non-hits since the previous hit
 *                         (for the first hit, since word 0); cell r counts gaps
 *                         of length r < t, cell t those of length >= t
 *                         (1 <= t <= 1024); words after the last hit close none. */
#define PRAND_TEST_FREQUENCY 0
#define PRAND_TEST_SERIAL 1
#define PRAND_TEST_GAP 2
typedef struct {
    int32_t kind;   /* PRAND_TEST_* */
    uint32_t bits;  /* frequency, serial */
    uint32_t t;     /* gap */
    uint32_t pad;
    uint64_t lo;    /* gap */
    uint64_t hi;    /* gap */
} prand_test_t;

/* Number of cells of a test, or 0 if its parameters are out of range. */
uint32_t prand_test_cells(const prand_test_t *test);

/* The cells' counts over dev_words[0..n): dev_counts (caller-owned device
 * memory, prand_test_cells() uint64 entries, 8-byte aligned) is overwritten.
 * dev_words: n words in device memory, 4-byte aligned (16-byte alignment gives
 * vector loads).  n < 2^40.  Asynchronous on `stream`; the gap test takes
 * stream-ordered scratch (cudaMallocAsync) of 16 bytes per 2^13 words.
 * Errors: PRAND_ERR_ARG, PRAND_ERR_ALIGN, PRAND_ERR_NOMEM, PRAND_ERR_CUDA. */
prand_status_t prand_test_counts(const prand_test_t *test, const uint32_t *dev_words, uint64_t n,
                                 uint64_t *dev_counts, prand_stream_t stream);

/* Pearson's chi-square statistic of host_counts (the counts of `test` over n
 * words) against the cells' expectations under the uniform hypothesis, and
 * its upper tail probability with (cells - 1) degrees of freedom:
 *   frequency  n / 2^bits per cell;
 *   serial     floor(n / 2) / 4^bits per cell;
 *   gap        G p (1 - p)^r for r < t and G (1 - p)^t, G = the number of
 *              gaps (the counts' sum), p = (hi - lo) / 2^32.
 * The tail probability is that of the chi-square law, valid when every
 * expectation is large (say >= 5); a p-value outside [1e-3, 1 - 1e-3] is the
 * paper's threshold for a suspicious result (Secs. 3-4).  Any output pointer may
 * be NULL.  Errors: PRAND_ERR_ARG (invalid test, n too small for one cell). */
prand_status_t prand_test_evaluate(const prand_test_t *test, uint64_t n, const uint64_t *host_counts, double *chi2,
                                   double *dof, double *pvalue);

/* Upper tail probability of the chi-square law with dof degrees of freedom at
 * x (x >= 0, dof > 0): the regularized incomplete gamma function Q(dof/2, x/2),
 * by its power series below x/2 < dof/2 + 1 and its continued fraction above
 * (evaluated by the modified Lentz method).  Returns NaN for invalid
 * arguments. */
double prand_chi2_sf(double x, double dof);

/* ---- Host SIMD generation (the paper's SSE realisations, Sec. 2 and Table 6,
 * restated for today's host vector units; no GPU involved) ----
 * MT19937, MRG32K3A or LFSR113 outputs of n_streams streams computed on the
 * host: host_states holds n_streams states in the one-struct-per-stream
 * layouts of prand_device.h (prand_mt19937_state, prand_mrg32k3a_state,
 * prand_lfsr113_state; e.g. from prand_export_states), advanced in place by
 * n_per_stream outputs; host_out[j * n_per_stream + i] = output i of stream j
 * as `dtype` (PRAND_DTYPE_U32 / _F32 / _F64), the same values prand_generate_*
 * writes for a handle holding those states.  MT19937 vectorises each stream's
 * twist four words at a time, LFSR113 four streams per vector, MRG32K3A two
 * streams per vector of exact double-precision products.  n_threads: host
 * threads the streams are spread over (0: one per hardware thread).  Returns
 * after the outputs are written.  host_states and host_out are caller-owned
 * host memory (host_out aligned to the element size, host_states to 4 bytes).
 * Errors: PRAND_ERR_ARG (another generator, unknown dtype, null pointer with
 * work to do, negative n_threads, size overflow), PRAND_ERR_ALIGN,
 * PRAND_ERR_STATE (an MT19937 state whose index exceeds 624). */
prand_status_t prand_host_generate(prand_gen_t gen, int32_t dtype, void *host_states, uint64_t n_streams,
                                   void *host_out, uint64_t n_per_stream, int32_t n_threads);

/* No counterpart in the paper.  MRG32K3A u32 generation that allocates no
 * memory, for callers that cannot call cudaMalloc: code that owns all device
 * memory through its own allocator or a fixed budget (a framework's caching
 * allocator, a long-running service), or that runs where an allocation would
 * synchronise the device or is not allowed.
 * dev_state: the caller's states of n_streams MRG32K3A streams, structure of
 * arrays, 6 * n_streams uint32 words: word c of stream j at dev_state[c *
 * n_streams + j], c = x_n, x_{n-1}, x_{n-2}, y_n, y_{n-1}, y_{n-2} (the payload
 * layout prand_get_state writes for an MRG32K3A handle).  The states are
 * advanced in place by n_per_stream outputs.  dev_out as in prand_generate_u32.
 * Scratch: a fixed device array inside the library (1.5 MB of next states for
 * at most 65536 streams, plus an 18 KB jump table), kept by every GPU that
 * loads the library until the process exits.  n_streams above 65536 returns
 * PRAND_ERR_ARG.  The first call on a device sets that device up (looks up the
 * array addresses and fills the table with one launch it waits for), so make
 * the first call before any stream capture; a call after a device reset
 * (cudaDeviceReset) finds a new context and repeats the set-up.  The calls
 * after the first check the device's context and array addresses on the host
 * (no device work, no wait).  All calls share the scratch:
 * calls that overlap on the GPU (different streams, or different host threads)
 * race and must be serialised by the caller.  Asynchronous on `stream` after
 * the first call.  Errors: PRAND_ERR_ARG, PRAND_ERR_ALIGN, PRAND_ERR_CUDA. */
prand_status_t prand_mrg32k3a_generate_u32_noalloc(uint32_t *dev_state, uint64_t n_streams, uint32_t *dev_out,
                                                   uint64_t n_per_stream, prand_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* PRAND_H */
