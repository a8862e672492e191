/*
 * sps.h - C ABI of libsps, a GB300 (sm_103a) library that applies quantum gate
 * streams to a state held only as its nonzero (basis label, amplitude) pairs.
 *
 * Method: arXiv 2105.01533, "Leveraging state sparsity for more efficient
 * quantum simulations".
 *   Sec. 3    the state sum_b alpha_b |b> is stored as unordered (label b,
 *             amplitude alpha_b) pairs with alpha_b != 0.
 *   Sec. 2.1  |i> = |i_{n-1}> (x) ... (x) |i_0>: qubit k is bit k of a label;
 *             gate matrices; CU = |0><0| (x) 1 + |1><1| (x) U.
 *   Sec. 3.1  gates with two nonzeros per row act on a label pair (b, b') by a
 *             2x2 matrix (Eq. 2); the result goes to a new container.
 *   Sec. 3.2  runs of gates with one nonzero per row (phases, permutations)
 *             compose as f1(b) f2(g1(b)) |g2(g1(b))> and are applied in one pass.
 *
 * Conventions for every entry point:
 *   - Labels are 128-bit: key_lo holds qubits 0..63, key_hi qubits 64..127.
 *     States of <= 63 qubits are stored with 64-bit labels; key_hi reads as 0.
 *   - Amplitudes are IEEE binary64 (re, im) pairs.
 *   - Pointers named "host or device" may point to pageable host memory,
 *     pinned host memory or device memory of the state's device (unified
 *     addressing decides); all others are host pointers unless stated.
 *   - The library owns all device memory it allocates (see sps_set_allocator).
 *   - Entry points return an sps_status; SPS_OK is 0. They never abort the
 *     process and never leave a kernel spinning: every wait inside a kernel is
 *     bounded and turns into an error code.
 *   - A state is bound to the CUDA stream given at creation; all its work is
 *     ordered on that stream. One state must not be used from two host threads
 *     at once; distinct states are independent.
 */
#ifndef SPS_H
#define SPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sps_status {
  SPS_OK = 0,
  SPS_ERR_ARG = 1,         /* bad argument or gate record (nothing was enqueued) */
  SPS_ERR_CAPACITY = 2,    /* the state would exceed its capacity, or an output
                              buffer is too small */
  SPS_ERR_TABLE_FULL = 3,  /* the branching hash table hit its probe limit */
  SPS_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  SPS_ERR_OOM = 5,         /* device allocation failed */
  SPS_ERR_NO_DEVICE = 6,   /* no usable CUDA device */
  SPS_ERR_TIMEOUT = 7      /* a device-side wait gave up (a grid barrier that
                              not every block reached within seconds) */
} sps_status;

/* Gate codes (sps_gate.op). Every gate takes any number of controls in
 * sps_gate.cmask (Sec. 2.1 controlled gates); a control must not coincide with
 * a target. Matrices are given in the basis (|0>, |1>) of the target.
 *   one nonzero per row (Sec. 3.2 phase/permutation gates):
 *     X [[0,1],[1,0]]   Y [[0,-i],[i,0]]   Z diag(1,-1)   S diag(1,i)
 *     SDG diag(1,-i)    T diag(1,e^{i pi/4})   TDG diag(1,e^{-i pi/4})
 *     P(theta) diag(1,e^{i theta})  (one control: controlled phase CP)
 *     RZ(theta) = exp(-i theta Z/2) = diag(e^{-i theta/2}, e^{i theta/2})
 *   two nonzeros per row (Sec. 3.1, Eq. 2):
 *     H sqrt(0.5)[[1,1],[1,-1]]
 *     RX(theta) = exp(-i theta X/2), RY(theta) = exp(-i theta Y/2)
 *     GIVENS(theta) on qubits (p = t0, q = t1): on the span of the label with
 *       bit p = 0, bit q = 1 (first) and the label with bit p = 1, bit q = 0
 *       (second) it acts by [[cos theta, -sin theta], [sin theta, cos theta]];
 *       labels with bit p == bit q are unchanged (number conserving).
 */
typedef enum sps_op {
  SPS_OP_X = 1, SPS_OP_Y = 2, SPS_OP_Z = 3, SPS_OP_S = 4, SPS_OP_SDG = 5,
  SPS_OP_T = 6, SPS_OP_TDG = 7, SPS_OP_P = 8, SPS_OP_RZ = 9,
  SPS_OP_H = 10, SPS_OP_RX = 11, SPS_OP_RY = 12, SPS_OP_GIVENS = 13
} sps_op;

/* One gate, 32 bytes, little-endian. */
typedef struct sps_gate {
  uint8_t op;          /* sps_op */
  uint8_t reserved0;   /* must be 0 */
  uint16_t t0;         /* target qubit (GIVENS: p) */
  uint16_t t1;         /* GIVENS: q; otherwise ignored */
  uint16_t reserved1;  /* must be 0 */
  uint64_t cmask[2];   /* control qubits: bit k of cmask[0] = qubit k,
                          bit k of cmask[1] = qubit 64 + k */
  double theta;        /* angle in radians (P, RZ, RX, RY, GIVENS) */
} sps_gate;

typedef struct sps_state sps_state; /* opaque, owned by the library */

/* Device memory hook. alloc(ctx, bytes, stream) returns a device pointer
 * aligned to >= 256 bytes or NULL (a pointer that is not so aligned is
 * released at once and counts as a failed allocation: SPS_ERR_OOM);
 * release(ctx, ptr, bytes, stream) frees it.
 * Both are called on the thread that calls into the library, with the
 * state's stream. Passing NULL for both restores the built-in allocator
 * (cudaMallocAsync on the state's stream). Affects states created afterwards. */
typedef void* (*sps_alloc_fn)(void* ctx, size_t bytes, void* stream);
typedef void (*sps_free_fn)(void* ctx, void* ptr, size_t bytes, void* stream);
sps_status sps_set_allocator(sps_alloc_fn alloc, sps_free_fn release, void* ctx);

/* Creates |0...0> on nqubits qubits (1..127) with room for `capacity`
 * nonzeros (>= 1) on the current CUDA device. `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream). The state keeps two label/amplitude
 * buffers of `capacity` entries (32 bytes each, 24 with 64-bit labels) and a
 * branching table of 32-byte slots (see sps_set_option). *out receives the
 * handle. Errors: SPS_ERR_ARG, SPS_ERR_OOM, SPS_ERR_CUDA, SPS_ERR_NO_DEVICE. */
sps_status sps_create(uint32_t nqubits, uint64_t capacity, void* cuda_stream,
                      sps_state** out);

/* Resets the state to |0...0> (no host wait). Also clears a pending
 * device-side error. The reset is recorded and carried out by the next call
 * that uses the state, in stream order: an sps_apply whose first pass is an
 * expansion (SPS_OPT_EXPAND) starts from |0...0> in that pass's own launch
 * (if that pass fails, the state is |0...0>); any other call enqueues the
 * reset first. */
sps_status sps_reset(sps_state* s);

/* Frees the state's device memory (after its stream's pending work). NULL ok. */
void sps_destroy(sps_state* s);

/* Applies `ngates` gates (host array, copied before return) in order, as one
 * batch: each maximal run of one-nonzero-per-row gates becomes one in-place
 * per-element pass (Sec. 3.2; a run is cut after SPS_OPT_MAX_FUSED_OPS gates or
 * when its P / RZ gates would need more than 61 phase slots, P taking one and
 * RZ two), each two-nonzero gate one branching pass
 * (Sec. 3.1) after which entries with re*re + im*im < prune_eps^2 (strict) or
 * exactly zero are dropped. prune_eps >= 0.
 * The call only enqueues work on the state's stream. Records are validated on
 * the host first: on a bad record it returns SPS_ERR_ARG, sets *failed_gate
 * (if not NULL) to its index and enqueues nothing. Errors found on the device
 * (SPS_ERR_CAPACITY, SPS_ERR_TABLE_FULL) are reported by the next sps_sync /
 * sps_nnz / sps_get_amplitudes / sps_probability; passes after the failing one
 * are skipped and the state is left exactly as it was before the failing pass. */
sps_status sps_apply(sps_state* s, const sps_gate* gates, size_t ngates,
                     double prune_eps, size_t* failed_gate);

/* Waits for the state's stream. Returns the first device-side error since the
 * last sync (and clears it, so the state is usable again, holding the result
 * of the last pass that succeeded). If failed_gate is not NULL and an error is
 * returned, it receives the index of the first gate of the failing pass within
 * the gate array of the sps_apply call that enqueued it. */
sps_status sps_sync(sps_state* s, size_t* failed_gate);

/* Synchronises like sps_sync and writes the number of stored nonzeros. */
sps_status sps_nnz(sps_state* s, uint64_t* nnz);

/* Synchronises like sps_sync and writes the nonzero-amplitude updates done
 * since creation or the last sps_reset: every applied gate counts the number
 * of nonzeros before it (passes skipped after an error count nothing). */
sps_status sps_get_updates(sps_state* s, uint64_t* updates);

/* Synchronises, then copies the state out in unspecified order: entry i is
 * (key_hi[i], key_lo[i], re[i], im[i]). Each pointer is host or device memory
 * of at least `cap` elements; key_hi may be NULL. *nnz_out receives the count;
 * if it exceeds cap nothing is copied and SPS_ERR_CAPACITY is returned. */
sps_status sps_get_amplitudes(sps_state* s, uint64_t* key_hi, uint64_t* key_lo,
                              double* re, double* im, uint64_t cap, uint64_t* nnz_out);

/* Replaces the state by n entries (host or device arrays; key_hi may be NULL
 * for all-zero high words). Labels must be distinct and use only qubits below
 * nqubits; amplitudes are taken as given. Errors: SPS_ERR_CAPACITY if
 * n > capacity, SPS_ERR_ARG on a label outside the qubit range. */
sps_status sps_set_amplitudes(sps_state* s, const uint64_t* key_hi, const uint64_t* key_lo,
                              const double* re, const double* im, uint64_t n);

/* Synchronises, then writes *p = sum of |alpha_k|^2 over stored labels k with
 * (k & mask) == value (mask/value: two words as in sps_gate.cmask). The sum is
 * formed in a fixed order for a given state layout, so it is reproducible. */
sps_status sps_probability(sps_state* s, const uint64_t mask[2], const uint64_t value[2],
                           double* p);

/* As sps_probability, but only enqueues: the sum is written to *out (pinned
 * host memory or device memory, owned by the caller, valid until the stream
 * has passed this point, e.g. until the next sps_sync) in stream order after
 * every pass enqueued before. With a pending device-side error it is the sum
 * over the last good state; the error is reported by the next sps_sync. */
sps_status sps_probability_async(sps_state* s, const uint64_t mask[2], const uint64_t value[2],
                                 double* out);

/* Registers a readout condition (mask, value as in sps_probability), or
 * clears it (both NULL). While it is set, an sps_apply whose last launch is
 * the compiled expansion form (a circuit that starts from a reset with an
 * expansion and a compiled phase/permutation run, SPS_OPT_BITSLICE_JIT) also
 * forms that condition's probability in the same launch, as the outputs are
 * stored; a later sps_probability or sps_probability_async with the same
 * condition, before any call that changes the state, then copies that sum
 * instead of launching the readout (counted in sps_counters.fused_readouts).
 * Other conditions, conditions testing fewer of the launch's label bits than
 * SPS_OPT_READOUT_MIN_PLANES (default 8, unless no label can match), and states
 * changed by other launches take the readout kernel as before. The fused sum is formed in a fixed order too (per block
 * of the launch, then over blocks in block order), which differs from the
 * readout kernel's, so the two may differ in the last bits. Allocates a few
 * KB of device memory on first use. Errors: SPS_ERR_ARG (one of mask, value
 * NULL), SPS_ERR_OOM. */
sps_status sps_set_readout(sps_state* s, const uint64_t mask[2], const uint64_t value[2]);

/* Applies exp(-i theta/2 P) for a Pauli string P (Sec. 3 lists Pauli
 * exponentials among the simulator's operations; Sec. 2.1 defines X, Y, Z and
 * R_P(theta) = exp(-i theta P / 2)). x[2] marks the qubits whose factor is X or
 * Y, z[2] those whose factor is Z or Y (Y where both are set; two words as in
 * sps_gate.cmask); cmask[2] are controls, disjoint from the string. With
 * P|j> = i^nY (-1)^popcount(j & z) |j ^ x> (nY = number of Y factors), a label
 * j with every control set goes to cos(theta/2)|j> - i sin(theta/2) P|j>.
 * A string with X or Y factors is one branching pass on the pairs (j, j ^ x)
 * (Sec. 3.1), pruned with prune_eps; a string of Z factors only is diagonal
 * and runs as a fused run (a CNOT ladder onto one z qubit, Rz, the ladder
 * undone). Enqueues only, like sps_apply; counts as one gate for the update
 * counter (the diagonal form counts its ladder). Errors: SPS_ERR_ARG for an
 * empty string, masks beyond nqubits, controls on the string or a non-finite
 * theta; device errors as for sps_apply (the failing gate is reported as 0). */
sps_status sps_pauli_exp(sps_state* s, const uint64_t x[2], const uint64_t z[2],
                         const uint64_t cmask[2], double theta, double prune_eps);

/* Measures qubit `qubit` in the computational basis and collapses the state
 * (Sec. 2.1: outcome b has probability sum |alpha_k|^2 over the labels whose
 * bit `qubit` is b, and the state is projected onto those labels; Sec. 3 lists
 * measurements among the simulator's operations). p0 and p1 are those sums
 * over the current state, formed on the device in a fixed order; the outcome is
 * 1 iff r * (p0 + p1) < p1, with r in [0, 1) drawn by the caller; labels
 * showing the other value are removed and the kept amplitudes are divided by
 * sqrt(p_outcome), so the state has norm 1 afterwards. Only enqueues: out[0] =
 * outcome (0.0 or 1.0) and out[1] = p_outcome / (p0 + p1) are written to `out`
 * (2 doubles of pinned host or device memory, caller-owned, valid until the
 * stream passes this point) in stream order. An empty state stays empty
 * (outcome 0, probability 0). Counts as one gate in sps_get_updates.
 * Errors: SPS_ERR_ARG for qubit >= nqubits or r outside [0, 1) (nothing is
 * enqueued); a pending device error skips it and is reported by sps_sync. */
sps_status sps_measure(sps_state* s, uint32_t qubit, double r, double* out);

/* Tuning options (see sps_set_option). */
typedef enum sps_option {
  SPS_OPT_LOAD_FACTOR_PCT = 1, /* target branching-table load, 10..90 (default 50) */
  SPS_OPT_PROBE_LIMIT = 2,     /* max slots probed per insert, >= 1 (default: table size) */
  SPS_OPT_BLOCK_THREADS = 3,   /* threads per block of the per-element kernels: 128 or
                                  256 (default 256) */
  SPS_OPT_MAX_FUSED_OPS = 4,   /* longest op list of one fused pass, 1..512 (default 512) */
  SPS_OPT_COOP_WIDTH = 5,      /* lanes probing one insert together: 1, 2, 4 or 8 */
  SPS_OPT_PROFILE = 6,         /* 1: time every kernel launch with CUDA events on the
                                  state's stream and log its entry counts; 0: off */
  SPS_OPT_BITSLICE_MIN_OPS = 7, /* fused passes with at least this many ops run
                                  bit-sliced (labels as bit-planes, 32 entries per
                                  logic op); 0 = never (default 8) */
  SPS_OPT_SMALL_RUN_CAP = 8,   /* consecutive passes whose nonzero bound stays at
                                  most this (<= 2048, default 2048) run in one
                                  single-block launch with the state in shared
                                  memory; 0 = never */
  SPS_OPT_BITSLICE_MIN_NNZ = 9, /* ... and only when the nonzero bound before the
                                  pass is at least this (default 262,144) */
  SPS_OPT_BITSLICE_GROUPS = 11, /* groups of 32 entries per warp tile in the
                                  bit-sliced pass: even, 2..32; 0 = chosen from
                                  the state size (default) */
  SPS_OPT_BRANCH_FORM = 10,    /* branching passes on the whole GPU: 0 default
                                  (gather), 1 scatter (labels emitted into a
                                  32-byte-slot table, FP64 atomic accumulation,
                                  separate prune/compact walk), 2 gather (each
                                  pair written once after a partner lookup in an
                                  index table; the insert-once rule of Sec. 3.1) */
  SPS_OPT_EXPAND = 12,         /* 1 (default): a run of up to 24 consecutive
                                  branching gates that act on every entry and
                                  whose flipped qubits are known to hold one
                                  value across the state (the host tracks this
                                  from sps_reset / sps_set_amplitudes through the
                                  gates) is applied in one expansion pass: no
                                  entry can meet a partner, so each entry writes
                                  its 2^d images with amplitude a times a product
                                  of matrix entries taken from per-8-gate tables
                                  (rounded once per table entry, so results match
                                  one-pass-per-gate within a few ulp rather than
                                  bit for bit; entries are pruned on the final
                                  amplitude). 0: one pass per gate */
  SPS_OPT_FOLD = 13,           /* 1 (default): in runs of phase/permutation gates,
                                  qubits known to hold one value (tracked as for
                                  SPS_OPT_EXPAND) are resolved on the host: gates
                                  with a control known 0 are dropped, known
                                  controls leave the condition, flips of known
                                  qubits are collected into one flip, and
                                  adjacent flips with one condition merge. The
                                  result is the same; the device walks fewer
                                  ops. 0: one op per gate */
  SPS_OPT_COMMUTE = 14,        /* 1: before compiling, rewrite each sps_apply
                                  stream with gate commuting queues (see
                                  sps_commute): H, Rx and Ry wait per qubit and
                                  cancel, merge or let phase/permutation gates
                                  pass. The state is the same up to rounding;
                                  pruning applies to the rewritten stream, and
                                  the update count counts the gates that run.
                                  0 (default): gate by gate */
  SPS_OPT_LAYER_GATES = 15     /* most branching gates in one layer pass, 1..4
                                  (default 4; 1 = one pass per gate): consecutive
                                  branching gates on pairwise disjoint qubits
                                  (targets and controls) run as one gather pass
                                  in which the member of each group with the
                                  largest selector pattern applies the gates in
                                  order to the group, with the same products,
                                  sums and pruning as one pass per gate (bit for
                                  bit). Not used inside one-block runs or with
                                  the scatter form */,
  SPS_OPT_EXPAND_WALK = 16     /* 1 (default): a run of phase/permutation gates
                                  right after an expansion pass (SPS_OPT_EXPAND)
                                  is applied by the expansion kernel to its
                                  outputs before they are stored: one launch,
                                  the state written once, the same values bit
                                  for bit (as the direct fused form; a run that
                                  takes the bit-sliced form, see
                                  SPS_OPT_BITSLICE_MIN_OPS, stays a pass of its
                                  own). 0: two passes */,
  SPS_OPT_FUSED_LABELS = 17    /* labels each thread of a direct fused pass walks
                                  together (sharing each op's decode): 1, 2, 4
                                  or 8; 0 (default) picks the most that still
                                  leave about four warps per SM */,
  SPS_OPT_AMP_ONLY = 18        /* 1 (default): a gather-form branching pass (one
                                  gate, or a layer pass) first tries the
                                  amplitude-only form: if every active label
                                  finds all members of its group and no value
                                  falls below eps or to zero, the labels stay
                                  in place and only amplitudes are written,
                                  with lookups in an index of all labels that
                                  stays valid while labels do not move (a pass
                                  that moves labels, or another use of the
                                  index table, makes the next attempt rebuild
                                  it). Branching passes on pairwise disjoint
                                  qubits (up to 32 gates) share one attempt,
                                  and a run of phase gates right after them is
                                  applied by it before the stores. The result
                                  is the same bit for bit (as the direct fused
                                  form, which such a phase run then takes).
                                  Where the form does not apply the usual
                                  kernels run, and the next 1, 2, 4 .. 64
                                  attempts are skipped. 0: never */,
  SPS_OPT_BITSLICE_JIT = 19    /* bit-sliced passes compiled for their run at run
                                  time (NVRTC; the op walk as straight-line code
                                  on registers, every row offset a constant; one
                                  compile per distinct run, cached for the
                                  process): 0 never, 1 (default) when the nonzero
                                  bound before the pass is at least 2^20, 2
                                  always. Where the runtime compiler is missing
                                  or a compile fails the general kernel runs;
                                  the results are the same */,
  SPS_OPT_PLAN_CACHE = 20      /* 1 (default): an sps_apply identical to the
                                  previous one (gates, threshold, options,
                                  starting knowledge, nonzero bound) reuses its
                                  compiled plan and the device copy of it; 0:
                                  every sps_apply compiles its gates and uploads
                                  the plan */,
  SPS_OPT_FALLBACK_CHAIN = 21  /* 1 (default): the passes an amplitude-only
                                  attempt stands in for are enqueued as one
                                  cooperative launch that returns at once when
                                  the attempt took the run and otherwise runs
                                  them in order with grid barriers (the same
                                  state as their separate launches); 0: each
                                  pass as its own launches */,
  SPS_OPT_READOUT_MIN_PLANES = 22 /* 8 (default): a registered readout
                                  (sps_set_readout) is summed by the compiled
                                  expansion launch only when it tests at least
                                  this many of the launch's label bits (or no
                                  label can match): a broad condition matches
                                  many outputs, whose amplitudes the launch
                                  would read back, and the readout kernel
                                  serves it better; 0..128 */
} sps_option;

/* Sets an option for subsequent sps_apply calls on this state. Errors:
 * SPS_ERR_ARG for an unknown option or out-of-range value. */
sps_status sps_set_option(sps_state* s, sps_option opt, int64_t value);

/* ---- Autotuner of the plain path ---------------------------------------------
 * sps_tune times whole steps of a circuit on the state (sps_reset, sps_apply,
 * sps_sync; wall clock, mean of `repeats` after one untimed step per setting)
 * and searches, one option at a time from the state's current settings:
 * SPS_OPT_LOAD_FACTOR_PCT (index-table load: 30, 50, 70), SPS_OPT_BITSLICE_GROUPS
 * (bit-sliced tile: 0, 8, 16, 32), SPS_OPT_FUSED_LABELS (0, 2, 4, 8) and
 * SPS_OPT_MAX_FUSED_OPS (fusion length: 128, 256, 512). The first three
 * change no result bit; the fusion length changes how phases of a run are
 * combined, so results agree to rounding. The best setting is left on the
 * state, which is left reset. A choice belongs to a size class: label words
 * kw (1 or 2) and log2peak = ceil(log2(projected peak nonzeros)), the peak
 * being min(capacity, the bound after the circuit's passes, doubling at every
 * branching gate). With cache_path non-null, a class already in that text file
 * takes its recorded choice without timing (from_cache = 1), and a newly timed
 * choice is appended as one line "sps-tune 1 kw=.. log2peak=.. load_factor_pct=..
 * bitslice_groups=.. fused_labels=.. max_fused_ops=.. ms=..". Errors:
 * SPS_ERR_ARG (bad record: as sps_apply; repeats outside 1..1000), or the
 * status of a failing step. */
typedef struct sps_tune_choice {
  uint32_t kw, log2peak;       /* the size class */
  uint32_t load_factor_pct;
  uint32_t bitslice_groups;
  uint32_t fused_labels;
  uint32_t max_fused_ops;
  uint32_t from_cache;         /* 1: taken from the cache file, not timed */
  float ms;                    /* mean step time of the choice (as recorded) */
} sps_tune_choice;

sps_status sps_tune(sps_state* s, const sps_gate* gates, size_t ngates, double prune_eps,
                    uint32_t repeats, const char* cache_path, sps_tune_choice* out);

/* Host-only: the choice recorded for size class (kw, log2peak) in a tuning
 * cache file (the last valid line of the class). SPS_ERR_ARG if the file
 * cannot be read or holds no valid line for the class. */
sps_status sps_tune_cache_lookup(const char* path, uint32_t kw, uint32_t log2peak,
                                 sps_tune_choice* out);

/* Exercises the grid barrier that the cooperative fallback launch uses
 * between passes: 8 blocks meet at three barriers whose waits give up after
 * `spins` polls (about 256 ns each); block skip_block (>= 8: none) does not
 * arrive at the first, so the other blocks' waits run out. *result receives
 * the status the launch recorded: SPS_OK when every block arrived,
 * SPS_ERR_TIMEOUT when a wait ran out (the launch still ends; later barriers
 * pass at once). Uses its own scratch control block and stream. Errors:
 * SPS_ERR_ARG (spins 0, result NULL), SPS_ERR_NO_DEVICE, SPS_ERR_CUDA. */
sps_status sps_barrier_selftest(uint32_t skip_block, uint32_t spins, sps_status* result);

/* Per-state counters since creation (host-side bookkeeping, no sync). */
typedef struct sps_counters {
  uint64_t gates;            /* gates accepted by sps_apply */
  uint64_t fused_passes;     /* per-element phase/permutation passes enqueued */
  uint64_t branch_passes;    /* branching passes enqueued */
  uint64_t kernel_launches;  /* kernels enqueued by this state */
  uint64_t upload_bytes;     /* compiled plans copied host -> device by sps_apply */
  uint64_t fused_readouts;   /* probability readouts answered from a registered
                                readout's sum (sps_set_readout), no launch */
} sps_counters;
sps_status sps_get_counters(sps_state* s, sps_counters* out);

/* One profiled kernel launch (SPS_OPT_PROFILE). kind: 1 fused phase /
 * permutation pass, 2 scatter emit, 3 scatter compaction, 4 small-state run
 * (several passes in one block), 5 gather index build, 6 gather emit,
 * 7 expansion pass (SPS_OPT_EXPAND; nops = gates), 8 measurement (sums and
 * collapse, timed together), 9 label index of amplitude-only passes
 * (SPS_OPT_AMP_ONLY; n_in 0 when the index was still valid or the attempt is
 * skipped), 10 amplitude-only attempt (n_out 0 when it did not take the pass;
 * then kinds 5 and 6 follow with n_in > 0; they show n_in 0 when skipped),
 * 11 the attempted run's passes in one launch (SPS_OPT_FALLBACK_CHAIN; nops =
 * passes; n_in 0 when the attempt took the run), 12 probability readout
 * (sps_probability and sps_probability_async; n_in = n_out = entries read;
 * none when a registered readout's sum is copied instead).
 * n_in: entries the kernel read; n_out: entries in the state after it. flags: bit 0 the
 * pass permutes labels, bit 1 it changes amplitudes, bit 2 (kinds 7 and 10) the
 * launch also applied the phase/permutation run after the branching gates,
 * bit 3 (kind 1) bit-sliced form, bit 4 (kind 1) the form compiled for this
 * run (SPS_OPT_BITSLICE_JIT), bit 5 (kind 7) the launch also summed the
 * registered readout (sps_set_readout). label_bytes: 8 or 16. */
typedef struct sps_kernel_record {
  uint32_t kind;
  uint32_t pass_serial;
  float ms;
  uint32_t nops;
  uint64_t n_in;
  uint64_t n_out;
  uint32_t flags;
  uint32_t label_bytes;
} sps_kernel_record;

/* Synchronises, then moves up to `cap` records of profiled launches (oldest
 * first) into out[] and *n; records that do not fit stay queued. */
sps_status sps_profile_read(sps_state* s, sps_kernel_record* out, size_t cap, size_t* n);

/* Host-only: gate commuting queues (Sec. 3.3 and Fig. 1). Rewrites a gate list
 * into one that computes the same state: H, Rx and Ry gates (without controls)
 * wait in per-qubit queues (pending op Ry Rx H on the qubit, above a queue of
 * phase/permutation gates); an incoming gate is commuted down through the
 * queues of its qubits with H H = 1, Rx(a) Rx(b) = Rx(a+b), Ry likewise,
 * H Ry(t) = Ry(-t) H, X Ry(t) = Ry(-t) X, Z Ry(t) = Ry(-t) Z, Z Rx(t) = Rx(-t) Z,
 * X Rx = Rx X, X H = H Z and Z H = H X (controlled X and Z through H on the
 * target); where no identity applies, the qubit's queue is emitted after the
 * phase/permutation queue. Everything is emitted at the end. Writes up to cap
 * records to out and the count to *nout (SPS_ERR_CAPACITY if more than cap).
 * Errors: SPS_ERR_ARG with *failed_gate on a bad record. */
sps_status sps_commute(const sps_gate* gates, size_t ngates, uint32_t nqubits, sps_gate* out,
                       size_t cap, size_t* nout, size_t* failed_gate);

/* Host-only: compiles a gate list for an nqubits-qubit state and describes the
 * passes without touching a GPU, for a state of which nothing is known (so no
 * expansion passes). For pass i: kind[i] = 1 (fused phase /
 * permutation run) or 2 (branching gate), first_gate[i] = index of its first
 * gate, ops[i] = number of device ops in the pass. At most `cap` passes are
 * written; *npasses receives the total. max_fused_ops as in SPS_OPT_MAX_FUSED_OPS
 * (0 = default). Errors: SPS_ERR_ARG with *failed_gate on a bad record. */
sps_status sps_plan(const sps_gate* gates, size_t ngates, uint32_t nqubits,
                    uint32_t max_fused_ops, uint32_t* kind, uint64_t* first_gate,
                    uint32_t* ops, size_t cap, size_t* npasses, size_t* failed_gate);

/* ---- Batched circuits ---------------------------------------------------------
 * Many independent circuits, each from |0...0>, advanced by one persistent
 * kernel launch. Blocks take circuits from a queue ordered by estimated work
 * (largest first); a circuit whose capacity fits the shared-memory cap runs
 * with its state in shared memory, others on their own device buffers. Each
 * circuit's progress is kept on the device, so sps_batch_run may advance every
 * circuit by a bounded number of passes and be called again to resume.
 * Branching passes use the insert-once rule of Sec. 3.1 (gather form, no
 * amplitude atomics); results equal sps_apply's. */
typedef struct sps_batch sps_batch;

typedef struct sps_batch_config {
  uint32_t threads;        /* threads per block: 256, 512 or 1024 */
  uint32_t blocks_per_sm;  /* persistent blocks per SM: 1..4 */
  uint32_t smem_cap;       /* circuits with capacity <= this (power of two,
                              64..2048, or 0) keep their state in shared memory */
  uint32_t reserved;
} sps_batch_config;

/* Creates an empty batch bound to `cuda_stream` (NULL = legacy default). */
sps_status sps_batch_create(void* cuda_stream, sps_batch** out);
void sps_batch_destroy(sps_batch* b);

/* Adds one circuit (gates copied; validated like sps_apply, SPS_ERR_ARG with
 * *failed_gate on a bad record). capacity: 1..2^24 nonzeros. *index receives
 * its position. Circuits can only be added before the first run or reset. */
sps_status sps_batch_add(sps_batch* b, uint32_t nqubits, uint64_t capacity,
                         const sps_gate* gates, size_t ngates, double prune_eps,
                         uint32_t* index, size_t* failed_gate);

/* Enqueues one launch advancing every unfinished circuit by up to max_passes
 * passes (0 = to completion). The first call allocates device memory. */
sps_status sps_batch_run(sps_batch* b, uint32_t max_passes);

/* One step of the batch as a captured CUDA graph: every circuit reset to
 * |0...0>, then the persistent launch advancing each by up to max_passes
 * passes (0 = to completion), as sps_batch_reset + sps_batch_run enqueue
 * them. The first call (and the first after max_passes or the launch
 * configuration changed) captures the step on a private stream and
 * instantiates it; every call launches the graph on the batch's stream (one
 * graph launch per step). The results equal those of the two calls. Errors:
 * SPS_ERR_CUDA if the capture or the instantiation fails (nothing enqueued). */
sps_status sps_batch_run_graph(sps_batch* b, uint32_t max_passes);

/* Waits for the batch's stream and reads back every circuit's progress;
 * *unfinished (nullable) receives the number still to run. */
sps_status sps_batch_sync(sps_batch* b, uint32_t* unfinished);

/* After sps_batch_sync: status of circuit `index` (SPS_OK or SPS_ERR_CAPACITY
 * with *failed_gate the first gate of the failing pass; the state is then the
 * one before that pass), its nonzero count and whether it has finished. */
sps_status sps_batch_circuit_status(sps_batch* b, uint32_t index, sps_status* status,
                                    size_t* failed_gate, uint64_t* nnz, int* finished);

/* After sps_batch_sync: copies circuit `index`'s state out (host or device
 * pointers, key_hi nullable), like sps_get_amplitudes. */
sps_status sps_batch_get_amplitudes(sps_batch* b, uint32_t index, uint64_t* key_hi,
                                    uint64_t* key_lo, double* re, double* im, uint64_t cap,
                                    uint64_t* nnz_out);

/* Enqueues a reset of every circuit to |0...0> with no progress. */
sps_status sps_batch_reset(sps_batch* b);

sps_status sps_batch_set_config(sps_batch* b, const sps_batch_config* cfg);
sps_status sps_batch_get_config(sps_batch* b, sps_batch_config* cfg);

/* Autotuner: runs the whole batch to completion `repeats` times under each of
 * a fixed set of block sizes, blocks per SM and shared-memory caps, keeps the
 * fastest (timed with CUDA events on the batch's stream), writes it to *best
 * and *best_ms (nullable) and leaves the batch reset. */
sps_status sps_batch_tune(sps_batch* b, uint32_t repeats, sps_batch_config* best,
                          float* best_ms);

/* Number of circuits and of batched launches enqueued so far. */
sps_status sps_batch_counts(sps_batch* b, uint32_t* ncircuits, uint64_t* launches);

/* After sps_batch_sync: nonzero-amplitude updates done since the last reset,
 * summed over circuits (each applied gate counts the nonzeros before it). */
sps_status sps_batch_updates(sps_batch* b, uint64_t* total);

/* ---- Serving: continuous batching of requests ---------------------------------
 * A request is a circuit from |0...0> with a capacity (the most nonzeros its
 * state may hold). The server charges it for its projected peak instead when
 * that is smaller: min(capacity, the nonzero bound after its passes, starting
 * from 1 and doubling at every branching gate), which no state of the circuit
 * can exceed, so the result and any capacity error are those of the declared
 * capacity. Requests are admitted in arrival order while an active slot and
 * enough of the memory budget are free (small requests, projected peak <=
 * 65,536: 64 B per entry; large ones: 96 B per entry plus 4 MiB). Each
 * sps_server_tick admits what fits, advances every active request by at most
 * passes_per_tick passes (0 = to completion) - small requests together in one
 * batched launch on the server's stream, large ones each as a whole-GPU state
 * on its own stream, so their work overlaps on the device - waits for them,
 * and copies finished requests to host memory, releasing their device memory.
 * Large requests' states run without SPS_OPT_BITSLICE_JIT (their passes
 * arrive a tick at a time; a run-time compile per slice would cost more than
 * most requests). Results equal sps_apply's for the same circuit. */
typedef struct sps_server sps_server;

typedef struct sps_server_request_info {
  int state;               /* 0 pending, 1 active, 2 done */
  sps_status status;       /* SPS_OK or the device-side error of the request */
  size_t failed_gate;      /* with an error: first gate of the failing pass */
  uint64_t nnz;            /* when done */
  uint64_t submit_tick;    /* server tick count at submission, admission and */
  uint64_t admit_tick;     /* completion (ticks are counted by sps_server_tick) */
  uint64_t done_tick;
  int large;               /* 1: ran as a whole-GPU state */
  uint64_t updates;        /* when done: nonzero-amplitude updates it took */
} sps_server_request_info;

sps_status sps_server_create(uint64_t mem_budget_bytes, uint32_t max_active,
                             uint32_t passes_per_tick, void* cuda_stream, sps_server** out);
void sps_server_destroy(sps_server* s);

/* Queues a request (gates copied and validated; SPS_ERR_ARG with
 * *failed_gate on a bad record; SPS_ERR_CAPACITY if it could never fit the
 * budget). *id receives its handle. */
sps_status sps_server_submit(sps_server* s, uint32_t nqubits, uint64_t capacity,
                             const sps_gate* gates, size_t ngates, double prune_eps,
                             uint64_t* id, size_t* failed_gate);

/* One scheduling step (blocking). Counts after the step go to the nullable
 * outputs: requests active, still pending, and finished in this step. */
sps_status sps_server_tick(sps_server* s, uint32_t* n_active, uint32_t* n_pending,
                           uint32_t* n_done);

sps_status sps_server_poll(sps_server* s, uint64_t id, sps_server_request_info* info);

/* Ids of the requests that finished in the last tick (up to cap; *n gets
 * the count, SPS_ERR_CAPACITY if cap was too small). */
sps_status sps_server_completed(sps_server* s, uint64_t* ids, size_t cap, size_t* n);

/* Copies a finished request's state (host pointers; key_hi nullable) and
 * forgets the request. SPS_ERR_CAPACITY with *nnz_out set if cap is too small. */
sps_status sps_server_result(sps_server* s, uint64_t id, uint64_t* key_hi, uint64_t* key_lo,
                             double* re, double* im, uint64_t cap, uint64_t* nnz_out);

/* Ticks so far, batched launches enqueued, device bytes charged to requests. */
sps_status sps_server_stats(sps_server* s, uint64_t* ticks, uint64_t* launches,
                            uint64_t* bytes_in_use);

/* Allocation-free variant of one branching pass, for callers that must not
 * allocate device memory (a host framework that owns all device memory and
 * forbids library allocations, a service whose device footprint is fixed at
 * start-up, or code running inside an allocator callback). The paper has no
 * counterpart; it is an interface convenience.
 * Applies ONE two-nonzero gate (`gate`: SPS_OP_H, RX, RY or GIVENS, host
 * pointer) to the n_in entries in the caller's device arrays in_*, prunes as
 * sps_apply does (prune_eps), and writes the result to the caller's device
 * arrays out_* (out_cap entries each, not aliasing the inputs); *n_out (host)
 * receives the count. nqubits (1..127) fixes the label width: for <= 63
 * qubits in_hi/out_hi are ignored and may be NULL. Input labels must be
 * distinct and use only qubits below nqubits.
 * Scratch: a fixed array inside the library image, 8,391,776 bytes (262,144
 * table slots of 32 B and a 3,168-byte control block), held by every GPU that
 * loads the library until the process exits. It allocates nothing: no
 * cudaMalloc, cudaFree or allocating library call. Limit: n_in <= 65,536,
 * else SPS_ERR_CAPACITY before anything is launched.
 * Each call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, a host-side query), so a device reset between calls
 * does not leave a stale address behind.
 * Every call uses the same array and it keeps the last call's contents; each
 * call clears the part it needs first. Calls that overlap on the GPU (on
 * different streams, host threads or processes sharing a context) race on the
 * array and give wrong results: serialise them. The call synchronises
 * `cuda_stream` before returning.
 * Errors: SPS_ERR_ARG (bad gate or pointers, or an out_* array equal to its
 * in_* counterpart), SPS_ERR_CAPACITY (n_in too
 * large, or more than out_cap entries result; *n_out = 0),
 * SPS_ERR_TABLE_FULL, SPS_ERR_CUDA, SPS_ERR_NO_DEVICE. */
sps_status sps_branch_apply_static(const sps_gate* gate, uint32_t nqubits,
                                   const uint64_t* in_hi, const uint64_t* in_lo,
                                   const double* in_re, const double* in_im, uint64_t n_in,
                                   double prune_eps, uint64_t* out_hi, uint64_t* out_lo,
                                   double* out_re, double* out_im, uint64_t out_cap,
                                   uint64_t* n_out, void* cuda_stream);

/* Host-only: 1 if the runtime compiler used by SPS_OPT_BITSLICE_JIT is
 * available and compiles the specialised kernel of a small sample run for
 * sm_103a, else 0; `log` (nullable, cap bytes) receives "ok" or the
 * compiler's message. Needs no GPU. */
int sps_jit_selftest(char* log, size_t cap);

/* Measures, on the current device, the issue rates of the units the kernels
 * lean on, as operations per second (lane operations): rates[0] FP64 fused
 * multiply-add, rates[1] FP32 fused multiply-add, rates[2] three-input 32-bit
 * logic, rates[3] 32-bit integer multiply-add. Each rate comes from a timed
 * launch of independent dependent chains (about 20 ms in all); the device
 * buffer it needs (8 bytes per thread) is allocated and freed with cudaMalloc.
 * These are the denominators for kernels bound by FP64 or by instruction
 * issue rather than by memory bandwidth. The paper has no counterpart: it is a
 * measurement aid. Errors: SPS_ERR_ARG, SPS_ERR_NO_DEVICE, SPS_ERR_OOM,
 * SPS_ERR_CUDA. */
sps_status sps_device_rates(double rates[4]);

/* Static text for a status code. */
const char* sps_status_str(sps_status st);

#ifdef __cplusplus
}
#endif

#endif /* SPS_H */
