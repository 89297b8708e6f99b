/*
 * corr.h -- C ABI of the GB300 X-engine (libcorr.so).
 *
 * The X-engine of an FX correlator (Sec. 2.3 of the paper "Design and
 * Implementation of a Scalable Correlator Based on ROACH2+GPU Cluster for
 * Tianlai 96-Dual-Polarization Antenna Array") performs, for every frequency
 * channel c, conjugate multiplication and accumulation (CMAC) over all input
 * pairs:
 *
 *     V_c[i][j] = sum_t x_c,i(t) * conj(x_c,j(t)),   i >= j          (Eq. 2)
 *
 * over the lower triangle including the autos, N(N+1)/2 products per channel
 * (Eq. 1), integrated over many blocks (Sec. 2.4: ~4 s integrations), with a
 * full-Stokes output (abstract, Sec. 1).
 *
 * Conventions shared by every call:
 *   - Inputs: N = n_ant * n_pol, input index i = n_pol * antenna + pol
 *     (pol 0 = X, pol 1 = Y).
 *   - Samples: one byte per complex sample, 4-bit two's complement real part
 *     in the high nibble and imaginary part in the low nibble (Sec. 2.1's
 *     4-bit + 4-bit requantised F-engine output).  All 256 byte values are
 *     valid, -8 included.
 *   - Block layout: uint8 x[n_chan][N][block_len] (channel-major "corner
 *     turned" order, Sec. 2.1's Transpose module).
 *   - Visibility layout: int64 vis[n_chan][P][2], P = N(N+1)/2, pair index
 *     i(i+1)/2 + j for i >= j, element 0 = real, 1 = imaginary.
 *   - Stokes layout (n_pol == 2): int64 stokes[n_chan][A][4][2],
 *     A = n_ant(n_ant+1)/2, antenna-pair index p(p+1)/2 + q for p >= q,
 *     order I, Q, U, V with
 *         XX = V[2p][2q], YY = V[2p+1][2q+1], XY = V[2p][2q+1], YX = V[2p+1][2q]
 *         (p == q: XY = conj(V[2p+1][2p]))
 *         I = XX + YY, Q = XX - YY, U = XY + YX, V = -j (XY - YX)   (no 1/2).
 *   - All arithmetic is integer and exact: results do not depend on block
 *     order or launch configuration.
 *   - Device pointers are CUDA device (or managed) addresses owned by the
 *     caller; host pointers are ordinary host memory (pinned memory makes the
 *     copies faster).  `stream` is a cudaStream_t (NULL = legacy default).
 *   - Every call returns CORR_OK (0) or a negative CORR_E* code; on error
 *     nothing is enqueued.  corr_strerror() names the code.
 *   - Thread safety: one context may be used by one host thread at a time,
 *     with all its device calls on one stream.  Independent contexts are
 *     independent.
 */
#ifndef CORR_H
#define CORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CORR_OK 0
#define CORR_EINVAL (-1)   /* bad argument (size, pointer, alignment, n_pol) */
#define CORR_ENOMEM (-2)   /* device or host allocation failed */
#define CORR_ECUDA (-3)    /* a CUDA runtime or driver call failed */
#define CORR_EARCH (-4)    /* current device is not compute capability 10.3 */
#define CORR_ETIMEOUT (-5) /* a device-side wait ran out; results are void */
#define CORR_ESTATE (-6)   /* call not valid in the context's current state */
#define CORR_EBOUNDS (-7)  /* debug builds: an address check or a guard band failed */

/* Largest block_len accepted (Sec. 2.4's integrations are blocks of many
 * samples; 2^24 - 1 bounds the host-side sample counters of one block). */
#define CORR_MAX_BLOCK_LEN 16777215
/* Samples the tensor cores accumulate in fp32 before a fold into int64.  A
 * partial over L samples is bounded by 128 * L, an exactly representable
 * integer (< 2^24) for L <= 131071; longer blocks, and launches of several
 * blocks, are folded at least this often. */
#define CORR_FOLD_SAMPLES 131071
/* Largest input count N = n_ant * n_pol accepted. */
#define CORR_MAX_INPUTS 8192

typedef struct corr_ctx corr_ctx;
typedef struct corr_server corr_server;

/*
 * Creates a correlator for n_ant antennas with n_pol (1 or 2) polarisations,
 * n_chan channels and blocks of block_len samples per channel (Sec. 2.3; the
 * paper's system is n_ant = 96, n_pol = 2, n_chan = 1024 over 125 MHz,
 * Sec. 2.2).  Allocates the int64 integration buffer on the current device
 * (n_chan * P * 16 bytes, zeroed) and a few kilobytes of bookkeeping.
 * The CMAC kernel is chosen here: the all-shared-memory kernel by default;
 * CORR_CMAC_KERNEL=tm in the environment selects the TMEM-operand kernel
 * (up to 192 inputs), =pair the CTA-pair kernel (more than 256 inputs).
 * On success *out owns them until corr_destroy.
 * Errors: CORR_EINVAL (non-positive size, n_pol not 1/2, block_len above
 * CORR_MAX_BLOCK_LEN, N above CORR_MAX_INPUTS, out NULL), CORR_EARCH,
 * CORR_ENOMEM, CORR_ECUDA.
 */
int corr_create(int n_ant, int n_pol, int n_chan, int block_len, corr_ctx **out);

/*
 * Integrates one block: for every channel, every i >= j,
 *   acc[c][i(i+1)/2 + j] += sum_{t < block_len} x[c][i][t] * conj(x[c][j][t]).
 * d_block: device pointer to uint8[n_chan][N][block_len], 16-byte aligned.
 * Stream-ordered and asynchronous; d_block must stay valid and unchanged until
 * the stream has executed the call.
 * Errors: CORR_EINVAL (NULL ctx/d_block, misaligned d_block), CORR_ECUDA.
 */
int corr_push_block(corr_ctx *ctx, const uint8_t *d_block, void *stream);

/*
 * Integrates n_blocks blocks (d_blocks: host array of n_blocks device
 * pointers, each as for corr_push_block).  Equivalent to n_blocks calls of
 * corr_push_block, but up to 8 blocks share one launch and one fold into the
 * int64 buffer (fewer while 8 * block_len exceeds CORR_FOLD_SAMPLES; a block
 * longer than that is folded every CORR_FOLD_SAMPLES samples or fewer).  The
 * pointer array itself may be reused as soon as the call returns.
 * Errors: CORR_EINVAL (NULL ctx or array, n_blocks < 1, a NULL or misaligned
 * block pointer; nothing is enqueued), CORR_ECUDA.
 */
int corr_push_blocks(corr_ctx *ctx, const uint8_t *const *d_blocks, int n_blocks, void *stream);

/*
 * Ends the integration: writes the visibilities accumulated since the last
 * dump to d_vis (int64[n_chan][P][2]) if it is not NULL, the full-Stokes
 * products to d_stokes (int64[n_chan][A][4][2]) if it is not NULL, and zeroes
 * the integration buffer.  Stream-ordered and asynchronous.
 * Errors: CORR_EINVAL (NULL ctx; d_stokes given with n_pol == 1),
 * CORR_ECUDA.
 */
int corr_dump(corr_ctx *ctx, int64_t *d_vis, int64_t *d_stokes, void *stream);

/*
 * Host-buffer variants.  corr_push_block_host copies h_block
 * (uint8[n_chan][N][block_len] in host memory) into a context-owned device
 * staging slot and integrates it on `stream`; it returns once h_block has been
 * copied, so the caller may reuse it, while the correlation itself may still
 * be running (the copy of the next block overlaps it).  corr_dump_host dumps
 * into context-owned device buffers and copies them to h_vis / h_stokes
 * (either may be NULL), returning when the host buffers are filled.  The
 * staging and output buffers are allocated on first use and freed by
 * corr_destroy.
 * Errors: as the device variants, plus CORR_ENOMEM.
 */
int corr_push_block_host(corr_ctx *ctx, const uint8_t *h_block, void *stream);
int corr_dump_host(corr_ctx *ctx, int64_t *h_vis, int64_t *h_stokes, void *stream);

/*
 * Sizes: *vis_elems = n_chan * P * 2, *stokes_elems = n_chan * A * 8 (0 when
 * n_pol == 1), *samples_integrated = samples per channel pushed since the last
 * dump.  Any output pointer may be NULL.
 */
int corr_sizes(const corr_ctx *ctx, size_t *vis_elems, size_t *stokes_elems,
               long long *samples_integrated);

/*
 * Waits for `stream`, then reads the context's device status word.  Returns
 * CORR_OK, CORR_ETIMEOUT if a device-side wait ran out since the last
 * successful check (the integration is then void and should be dumped and
 * discarded), or CORR_ECUDA.  Clears the status word.
 */
int corr_check(corr_ctx *ctx, void *stream);

/*
 * Host-only view of the tile schedule for n_in inputs (no device needed).
 * cover, if not NULL, is uint8[n_in][n_in] and receives +1 for every element
 * (i, j) that the schedule's MMAs fold into the integration buffer (the lower
 * triangle, each element exactly once).  *n_units receives the work units per
 * channel and *issued_cmacs the complex MACs per channel per sample that the
 * MMAs issue (lower triangle plus the padding they also compute; the useful
 * count is n_in(n_in+1)/2).  Errors: CORR_EINVAL (n_in out of range).
 */
int corr_plan(int n_in, uint8_t *cover, int *n_units, long long *issued_cmacs);

/* Triangle covers (the tile schedule's shape; see corr_plan_cover).
 *   WINDOW: N <= 256.  Every unit stages all inputs once per chunk, and the
 *           64-input row tiles' strips share it, packed into 512 TMEM columns.
 *   STRIPS: N <= 256.  One unit per row tile t, staging inputs [0, 64(t+1)).
 *   PAIRS:  any N.  Pairs of row tiles against 256-column pieces of their
 *           strip; one CTA per unit.
 *   QUADS:  N > 256.  Blocks of 256 rows against 256-column pieces of their
 *           strip, each run by a pair of CTAs on two SMs (a 2-CTA cluster):
 *           each CTA stages 128 of the rows and half of the piece's columns,
 *           and the pair's M = 256 tensor-core MMAs share the columns.  On
 *           the diagonal the CTAs take row tiles 0 and 3, and 1 and 2, so
 *           that tiles 0 and 1 run against 128 columns only.
 *           Contexts use it only when CORR_CMAC_KERNEL=pair is set.
 * WINDOW and STRIPS fall back to PAIRS above 256 inputs, QUADS to PAIRS at
 * 256 and below.  CORR_CMAC_KERNEL=pair in the environment makes contexts of
 * more than 256 inputs use QUADS, =smem PAIRS. */
#define CORR_COVER_WINDOW 0
#define CORR_COVER_STRIPS 1
#define CORR_COVER_PAIRS 2
#define CORR_COVER_QUADS 3

/* As corr_plan, for the given cover.  Errors: CORR_EINVAL (n_in out of
 * range, unknown cover). */
int corr_plan_cover(int n_in, int cover, uint8_t *cover_out, int *n_units,
                    long long *issued_cmacs);

/*
 * Host-only view of how one launch's work is dealt to the GPU's
 * multiprocessors (no device needed).
 *   - A unit is (template, channel): one of the cover's n_units templates on
 *     one channel, over all n_blocks blocks of block_len samples.
 *   - Units are cut at 128-sample stage boundaries into items, and every CTA
 *     (at most `grid`) runs a contiguous run of items of about equal
 *     modelled cost.  That cost is the operand rows unpacked plus a fixed
 *     fold cost per item.  No item spans more than CORR_FOLD_SAMPLES / 128
 *     stages (1023): each item folds its fp32 partials into int64 once.
 *   - n_blocks: 1..8 (the blocks of one launch).
 *   - items, if not NULL, receives up to `cap` rows of 5 ints:
 *     (problem = 0, template, channel, first stage, stages).  Stage k of the
 *     launch is 128-sample stage k % ceil(block_len / 128) of block
 *     k / ceil(block_len / 128).
 *   - cta_first, if not NULL, receives grid + 1 ints: CTA b runs items
 *     [cta_first[b], cta_first[b + 1]), for b < *used_grid.
 *   - *n_items and *used_grid receive the totals.
 * Errors: CORR_EINVAL (sizes out of range, unknown cover, or cap < *n_items
 * with items given; *n_items is still set).
 */
int corr_plan_items(int n_in, int n_chan, int block_len, int n_blocks, int cover, int grid,
                    int *items, int cap, int *n_items, int *cta_first, int *used_grid);

/*
 * Visibilities of one block without any allocation.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory -- code inside a framework that owns the whole device memory
 * pool, and code on a real-time path where the implicit synchronisation of
 * cudaMalloc/cudaFree would stall queued work.
 *
 * Writes vis[c][i(i+1)/2 + j] = sum_t x[c][i][t] conj(x[c][j][t]) for one
 * block (no integration across calls, no Stokes) into d_vis
 * (int64[n_chan][P][2], overwritten), from d_block as for corr_push_block.
 * The kernel's scratch memory (its tile schedule and status word) lives in a
 * file-scope device array of CORR_STATIC_SCRATCH_BYTES that every GPU which
 * loads the library holds until the process exits; the call allocates nothing
 * on the device or the host.
 *   - Limits: n_ant * n_pol <= CORR_STATIC_MAX_INPUTS, block_len a multiple of
 *     16 (at most CORR_STATIC_MAX_BLOCK_LEN, one fold per call); d_block and
 *     d_vis 16-byte aligned.
 *     Anything else returns CORR_EINVAL before any work is enqueued.
 *   - The first call on a device looks up the array's device address and the
 *     device limits; make that first call before any stream capture.  With
 *     CUDA's default lazy module loading, that first lookup (or the first
 *     launch) also loads the library's device code on that device, which the
 *     driver allocates once, outside any framework's pool: make the first
 *     call at set-up, not on the path that must not allocate.  Later calls
 *     allocate nothing.
 *   - Each call enqueues a one-block set-up kernel that receives the tile
 *     schedule by value in its parameters and writes it into the array
 *     (nothing is copied from host memory), a memset of d_vis and the
 *     X-engine launch.
 *   - Every call shares the one array and leaves its contents behind: calls
 *     whose work overlaps on the GPU (other streams, other host threads) race
 *     on it; serialise them.
 *   - A device-side wait that runs out leaves d_vis incomplete and cannot be
 *     reported here (there is no context); callers that need that check use
 *     corr_create / corr_check.
 * Stream-ordered and asynchronous.  Errors: CORR_EINVAL, CORR_EARCH,
 * CORR_ECUDA.
 */
#define CORR_STATIC_SCRATCH_BYTES 4096
#define CORR_STATIC_MAX_INPUTS 256
#define CORR_STATIC_MAX_BLOCK_LEN 131056
int corr_xcorr_static(const uint8_t *d_block, int n_ant, int n_pol, int n_chan, int block_len,
                      int64_t *d_vis, void *stream);

/*
 * Corner turn (Sec. 2.1: the Transpose module that reorders the F-engine
 * output for the correlation), on the device:
 *     d_dst[c][i][t] = d_src[t][c][i]
 * for a block in F-engine order, uint8 [block_len][n_chan][n_in] (one
 * spectrum per time step), to the X-engine order of corr_push_block, uint8
 * [n_chan][n_in][block_len].  The call reads and writes every byte once.
 *   - Any sizes are accepted.
 *   - d_src and d_dst must be 4-byte aligned, must not overlap, and are
 *     owned by the caller.
 * Stream-ordered and asynchronous.  Errors: CORR_EINVAL (NULL or misaligned
 * pointer, non-positive size), CORR_ECUDA.
 */
int corr_corner_turn(const uint8_t *d_src, uint8_t *d_dst, int n_in, int n_chan, int block_len,
                     void *stream);

/*
 * As corr_push_block for a block in F-engine order, uint8
 * [block_len][n_chan][N] (d_src, 4-byte aligned): the Transpose step of
 * Sec. 2.1 and the correlation in one call.
 *   - When N is a multiple of 16, d_src is 16-byte aligned and the context
 *     runs the all-shared-memory CMAC kernel (the default; not with
 *     CORR_CMAC_KERNEL=tm or =pair), the CMAC kernel stages the block in this order
 *     itself: its TMA boxes are [128 samples][64 inputs] of one channel and
 *     the unpack transposes them on chip.  One launch; every byte is read
 *     once.
 *   - Otherwise the block is first corner-turned into a context-owned buffer
 *     (allocated on the first such call, freed by corr_destroy), then
 *     integrated: two launches.
 * d_src may be reused once the stream has executed the call.  Errors: as
 * corr_push_block, plus CORR_ENOMEM.
 */
int corr_push_block_tcn(corr_ctx *ctx, const uint8_t *d_src, void *stream);

/*
 * Failure-detection self-test.  Runs one CMAC launch over d_block (as for
 * corr_push_block) in which the accumulator-draining warps first wait for a
 * barrier that nothing ever completes.  That wait is bounded like every other
 * device-side wait: after timeout_ms (1..10000) it gives up, raises the
 * kernel's abort flag, and every role winds down.  The roles drain their own
 * copies and tensor-core work, free TMEM and set the context's status word.
 * Nothing is folded, so the integration buffer and the sample count are
 * unchanged.  The next corr_check returns CORR_ETIMEOUT and clears the status;
 * the context stays usable.  No fault, trap or unbounded wait is involved.
 * Errors: CORR_EINVAL (NULL or misaligned pointer, timeout out of range),
 * CORR_ECUDA.
 */
int corr_selftest_timeout(corr_ctx *ctx, const uint8_t *d_block, int timeout_ms, void *stream);

/* Number of kernel launches the context has enqueued (pushes and dumps). */
long long corr_launch_count(const corr_ctx *ctx);

/*
 * Counters of a context, kept on the host as calls are enqueued (nothing is
 * read from the device).  An integration (Sec. 2.4) is the blocks pushed
 * between two dumps.
 */
typedef struct corr_stats {
  long long blocks_pushed;   /* blocks integrated since corr_create */
  long long samples_total;   /* samples per input integrated since corr_create */
  long long samples_pending; /* samples per input in the integration in progress */
  long long dumps;           /* completed corr_dump / corr_dump_host calls */
  long long launches;        /* kernel launches enqueued (as corr_launch_count) */
} corr_stats;

/* Fills *out.  Errors: CORR_EINVAL (ctx or out NULL). */
int corr_get_stats(const corr_ctx *ctx, corr_stats *out);

/*
 * Checkpoint of the integration in progress.  The accumulators are integers,
 * so an integration resumed from a snapshot ends bit-identical to one that
 * never stopped.
 *
 * corr_snapshot waits for `stream`, then copies the int64 accumulators to
 * h_acc (caller-owned host memory of vis_elems int64, the layout of
 * corr_dump's visibilities: [n_chan][P][2]) and the integration's sample count
 * to *samples.  The context is unchanged.
 *
 * corr_restore replaces the integration in progress of `ctx` with a snapshot
 * taken from a context of the same shape (this one or another, in this
 * process or an earlier one): it copies h_acc to the accumulators on `stream`,
 * waits for the copy, and sets the integration's sample count to `samples`.
 *
 * Errors: CORR_EINVAL (NULL pointers, samples < 0), CORR_ECUDA.
 */
int corr_snapshot(corr_ctx *ctx, int64_t *h_acc, long long *samples, void *stream);
int corr_restore(corr_ctx *ctx, const int64_t *h_acc, long long samples, void *stream);

/*
 * Debug builds.  Compiling the library with CORR_DEBUG defined (the Python
 * build's debug variant, libcorr_debug.so) adds checks that cost time and
 * change no result:
 *   - every int64 atomic add of the CMAC kernels' fold and every element the
 *     dump touches is checked against its integration buffer; an address
 *     outside it is skipped and recorded;
 *   - a context's integration buffer gets a guard band of 4096 bytes on each
 *     side, filled with 0xA5 at creation; corr_check compares both bands with
 *     the pattern before it reads the status word.
 * A recorded failure makes the next corr_check (corr_batch_check for the
 * address checks of a batch) return CORR_EBOUNDS, which takes precedence over
 * CORR_ETIMEOUT.  Release builds carry none of this code.
 *
 * corr_debug_build returns 1 in a debug build, else 0.
 * corr_debug_corrupt_guard overwrites one byte in the middle of the guard
 * band before (side 0) or after (side 1) the integration buffer, from the
 * host, so that a test can see corr_check report it.  Errors: CORR_EINVAL,
 * CORR_ESTATE (release build), CORR_ECUDA.
 */
int corr_debug_build(void);
int corr_debug_corrupt_guard(corr_ctx *ctx, int side);

/*
 * Batches: many independent correlators in shared launches.
 *
 * The paper's system runs one X-engine per server and pipeline instance,
 * each on its own array (Sec. 2.2-2.3).  A batch holds n_inst such
 * correlators, each with its own n_ant, n_pol, n_chan and block_len.
 *   - Each instance has its own int64 integration buffer, sized and laid out
 *     as a context's.
 *   - One corr_batch_push integrates one block of every instance.
 *   - The units of all instances are dealt to the multiprocessors of one
 *     persistent launch per shared-memory layout, so instances with few
 *     channels fill the gaps left by large ones.
 *   - With CORR_BATCH_AUTOTUNE, each distinct (input count, block length
 *     rounded up to a power of two) gets its triangle cover by timing one
 *     launch of every candidate cover on a synthetic problem of that size.
 *     The choice is cached for the process.
 *   - Results are bit-identical to one context per instance: every sum is
 *     an exact integer.
 */
#define CORR_BATCH_AUTOTUNE 1
typedef struct corr_batch corr_batch;

/* Creates the batch: arrays of n_inst sizes (as for corr_create).
 * Allocates every integration buffer (zeroed) on the current device.
 * Errors: CORR_EINVAL (any size as for corr_create, unknown flag, NULL
 * array), CORR_EARCH, CORR_ENOMEM, CORR_ECUDA, CORR_ETIMEOUT (while tuning). */
int corr_batch_create(int n_inst, const int *n_ant, const int *n_pol, const int *n_chan,
                      const int *block_len, int flags, corr_batch **out);

/* Integrates one block of every instance.  d_blocks is a host array of n_inst
 * device pointers, instance k's block laid out as for corr_push_block with
 * that instance's sizes, 16-byte aligned.  Stream-ordered and asynchronous;
 * the blocks must stay unchanged until the stream has executed the call.
 * The pointer array may be reused at once.
 * Errors: CORR_EINVAL (NULL batch or array, a NULL or misaligned pointer;
 * nothing is enqueued), CORR_ECUDA. */
int corr_batch_push(corr_batch *b, const uint8_t *const *d_blocks, void *stream);

/* As corr_dump, for instance `inst` alone (its buffer is zeroed; the others
 * keep integrating).  Errors: CORR_EINVAL (inst out of range, d_stokes with
 * n_pol == 1, misaligned pointer), CORR_ECUDA. */
int corr_batch_dump(corr_batch *b, int inst, int64_t *d_vis, int64_t *d_stokes, void *stream);

/* As corr_sizes, for instance `inst`.  Errors: CORR_EINVAL. */
int corr_batch_sizes(const corr_batch *b, int inst, size_t *vis_elems, size_t *stokes_elems,
                     long long *samples_integrated);

/* Instance `inst`'s cover (CORR_COVER_*), its launch group, and the number of
 * launch groups (one CMAC launch each per push).  Any output may be NULL.
 * Errors: CORR_EINVAL. */
int corr_batch_info(const corr_batch *b, int inst, int *cover, int *group, int *n_groups);

/* As corr_check, for the batch's device status word. */
int corr_batch_check(corr_batch *b, void *stream);

/* Kernel launches the batch has enqueued (pushes and dumps). */
long long corr_batch_launch_count(const corr_batch *b);

/* Releases the batch.  The caller must have synchronised its streams.  NULL
 * is ignored. */
void corr_batch_destroy(corr_batch *b);

/* The autotuner's cached cover for (n_in, block_len), or -1 if none is cached
 * yet.  Host-only.  Errors: CORR_EINVAL (non-positive size). */
int corr_tuned_cover(int n_in, int block_len);

/* Releases everything the context owns.  The caller must have synchronised
 * every stream that used it.  NULL is ignored. */
void corr_destroy(corr_ctx *ctx);

/*
 * Serving: a loop that takes blocks of several arrays as they arrive on the
 * host and returns each completed integration's visibilities.
 *
 * The paper's system runs hashpipe threads around ring buffers: network
 * input, GPU correlation and output (Sec. 2.3).  corr_server_create starts
 * one worker thread that owns three CUDA streams, one each for
 * host-to-device copies, correlation and device-to-host copies, plus:
 *   - an arena of `arena_bytes` of device memory for block slots (first-fit
 *     allocation; blocks wait in arrival order while it is full, so the
 *     budget bounds the HBM in flight);
 *   - per array, a context (resident int64 accumulators) and a pinned host
 *     result buffer.
 *
 * Blocks carry (array, seq).  Integration k of an array holds sequence
 * numbers [k L, (k + 1) L), L = blocks_per_integration (1..64).  Blocks may
 * arrive in any order:
 *   - A block up to `window` - 1 integrations ahead of the current one is
 *     staged and held.
 *   - A block `window` or more integrations ahead closes the integrations it
 *     leaves behind.  A closed integration completes with the blocks it
 *     holds; the rest count as dropped.
 *   - Duplicates, and blocks of closed or finished integrations, are
 *     discarded and counted.
 * corr_server_flush closes every open integration.
 */
typedef struct {
  int n_ant, n_pol, n_chan, block_len;
  int blocks_per_integration;  /* L, 1..64 */
} corr_array_desc;

typedef struct {
  int array;
  long long integration;  /* k: sequence numbers [k L, (k + 1) L) */
  int n_blocks;           /* blocks integrated (L unless some were dropped) */
  uint64_t block_mask;    /* bit s: sequence number k L + s was integrated */
  const int64_t *vis;     /* int64[n_chan][P][2] in a server-owned pinned buffer, valid
                             until corr_server_release(array); NULL in dry mode */
  double t_first_arrival_ms, t_last_arrival_ms, t_done_ms; /* steady clock */
} corr_result;

typedef struct {
  long long submitted, integrated, duplicates, late, integrations, incomplete_integrations;
  double latency_p50_ms, latency_p99_ms, latency_max_ms; /* block arrival -> result ready */
  long long latency_samples;
  size_t arena_peak_bytes;
  int error; /* first error of the worker, CORR_OK if none */
} corr_server_info;

/* Dry mode: no device work at all (copies, pushes and dumps complete at once,
 * results carry no visibilities); the admission and ordering policy runs
 * unchanged, so it can be tested without a GPU. */
#define CORR_SERVER_DRY 1

/* Errors: CORR_EINVAL (sizes as for corr_create, L out of 1..64, window < 1,
 * arena smaller than the largest block, unknown flag), CORR_EARCH,
 * CORR_ENOMEM, CORR_ECUDA. */
int corr_server_create(int n_arrays, const corr_array_desc *arrays, size_t arena_bytes, int window,
                       int flags, corr_server **out);

/* Queues block `seq` of `array` (uint8[n_chan][N][block_len] in host memory,
 * pinned for full copy speed) and returns at once.  h_block must stay valid
 * and unchanged until the integration that holds it has been returned by
 * corr_server_poll, or the block was discarded, or the server is destroyed.
 * Errors: CORR_EINVAL (bad array, negative seq, NULL block outside dry mode),
 * or the worker's error. */
int corr_server_submit(corr_server *s, int array, long long seq, const uint8_t *h_block);

/* Moves up to max_results completed integrations into out[], oldest first,
 * waiting up to timeout_ms for the first.  Returns how many, or a negative
 * error (the worker's, or CORR_EINVAL). */
int corr_server_poll(corr_server *s, corr_result *out, int max_results, int timeout_ms);

/* The caller is done with the array's last result; its buffer may be reused
 * for the next integration (which is held back until then). */
int corr_server_release(corr_server *s, int array);

/* Closes every open integration (see above). */
int corr_server_flush(corr_server *s);

/* Counters and latency percentiles so far. */
int corr_server_stats(corr_server *s, corr_server_info *out);

/* Stops the worker, waits for the device, frees everything.  Results not yet
 * polled are lost.  NULL is ignored. */
void corr_server_destroy(corr_server *s);

/*
 * F-engine on the GPU (Sec. 2.1): polyphase filter bank, real FFT, EQ and
 * 4+4-bit requantisation of 8-bit ADC samples, written in the X-engine's
 * input order so the output feeds corr_push_block directly.
 *
 * For one input with samples x (a stream of (n_spectra + 3) * 2048 int8
 * values), spectrum k (0 <= k < n_spectra) is
 *     v_k[n] = sum_{j<4} h[2048 j + n] x[2048 (k + j) + n],      n < 2048
 *     X_k[c] = sum_n v_k[n] exp(-2 pi i n c / 2048),               c < 1024
 * with the 8192-tap prototype h[m] = w[m] sinc((m - 4096) / 2048), where
 * w[m] = 0.54 - 0.46 cos(2 pi m / 8191) is the Hamming window (the paper's
 * PFB size 2^11, 4 taps, Hamming window; FFT size 2^11).  With EQ gain
 * g[i][c] the output byte is
 *     out[c][i][k] = (q(g Re X) << 4) | (q(g Im X) & 15)
 * where q rounds half away from zero and clips to [-7, 7].  Arithmetic is
 * fp32, so a code can differ from the exact one only where g X lies within
 * the fp32 rounding error of a quantisation boundary.
 */
#define CORR_FENGINE_POINTS 2048
#define CORR_FENGINE_CHANNELS 1024
#define CORR_FENGINE_TAPS 4
typedef struct corr_fengine corr_fengine;

/* n_in inputs, n_spectra spectra per run; EQ gains start at 1.
 * Errors: CORR_EINVAL, CORR_EARCH, CORR_ENOMEM, CORR_ECUDA. */
int corr_fengine_create(int n_in, int n_spectra, corr_fengine **out);

/* Copies EQ gains float[n_in][1024] from host memory (synchronous). */
int corr_fengine_set_eq(corr_fengine *f, const float *h_eq);

/* d_adc: int8[n_in][(n_spectra + 3) * 2048] device samples (16-byte aligned);
 * d_out: uint8[1024][n_in][n_spectra] device (16-byte aligned), overwritten.
 * Stream-ordered and asynchronous.  Errors: CORR_EINVAL, CORR_ECUDA. */
int corr_fengine_run(corr_fengine *f, const int8_t *d_adc, uint8_t *d_out, void *stream);

/* As corr_fengine_run, but writes g X unquantised: float[1024][n_in][n_spectra][2]
 * (real, imaginary).  For inspection and tests. */
int corr_fengine_spectra(corr_fengine *f, const int8_t *d_adc, float *d_spec, void *stream);

void corr_fengine_destroy(corr_fengine *f);

/*
 * Dense tensor-core rate of the current GPU (a measurement helper for the
 * roofline of the CMAC kernel; the paper has no counterpart).  Launches one
 * CTA per SM; in each, `issuers` threads (1..4) issue `iters` x 4
 * back-to-back tcgen05.mma.kind::f8f6f4 instructions (E5M2 operands, fp32
 * accumulation, M = 128, N = n, K = 32) into their own TMEM accumulators,
 * with both operands in 128B-swizzled shared memory, or with A in TMEM when
 * a_from_tmem is 1.  The work is
 *     n_SM * issuers * iters * 4 * 2 * 128 * n * 32   floating-point ops;
 * the caller times the launch on `stream` (CUDA events).
 *   - n: multiple of 16 in [16, 256]; issuers * n (+ 32 with a_from_tmem)
 *     <= 512 TMEM columns; iters in [1, 10^7].
 *   - d_status: device int; bit 0 is set if the final wait for the MMAs ran
 *     out (2 s).  d_cycles: device int64[n_SM] or NULL; receives each CTA's
 *     clock64 cycles from its first MMA to the completion of its last.
 * Stream-ordered and asynchronous.  Errors: CORR_EINVAL, CORR_EARCH,
 * CORR_ECUDA.
 */
int corr_mma_rate(int n, int issuers, int iters, int a_from_tmem, int *d_status,
                  long long *d_cycles, void *stream);

/* Static string naming a CORR_* code. */
const char *corr_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* CORR_H */
