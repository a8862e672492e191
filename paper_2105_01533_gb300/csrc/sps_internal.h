// Internal types shared by the host compiler, the kernels and the C ABI layer
// of libsps. Nothing here is part of the public interface (include/sps.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "sps.h"

#ifndef __CUDACC__
#define __host__
#define __device__
#define __align__(n) alignas(n)
#endif

namespace sps {

// ---- compiled per-element op (Sec. 3.2) --------------------------------------
// A run of one-nonzero-per-row gates maps alpha_b |b> to f(b) alpha_b |g(b)>;
// composing gates is applying their ops in order to the running label:
//   if ((k & c) == c) {
//     sel  = (sbit == NO_SEL) ? 0 : bit sbit of k
//     cnt += sel ? a1 : a0                      // phase e^{i pi cnt / 4}
//     if (ph != NO_PH) acc *= phase[ph][sel]    // arbitrary-angle phase
//     k   ^= t                                  // permutation
//   }
// Phases are read before the flip, i.e. from the label the gate acts on.
constexpr uint8_t NO_SEL = 0xFF;
constexpr uint16_t NO_PH = 0xFFFF;

struct FOp {            // 48 bytes
  uint64_t c[2];        // condition mask: all these bits must be 1
  uint64_t t[2];        // xor mask applied when the condition holds
  uint8_t a0, a1;       // pi/4 steps added when sel = 0 / 1 (mod 8)
  uint8_t sbit;         // selector qubit or NO_SEL
  uint8_t kind;         // FOP_* flags, derived from the fields (set_fop_kind)
  uint16_t ph;          // index into the pass's phase pairs or NO_PH
  uint16_t reserved2;
  uint64_t reserved3;
};
static_assert(sizeof(FOp) == 48, "FOp layout");

// FOp::kind flags: which parts of the op do anything, so the per-entry walk
// skips the rest (the flags are uniform over a warp: every thread walks the
// same list).
constexpr uint8_t FOP_FLIP = 1;   // t != 0
constexpr uint8_t FOP_CNT = 2;    // a0 or a1 != 0
constexpr uint8_t FOP_PH = 4;     // ph != NO_PH
constexpr uint8_t FOP_SEL = 8;    // sbit != NO_SEL
constexpr uint8_t FOP_HI = 16;    // c or t touch qubits 64..127
inline void set_fop_kind(FOp& o) {
  o.kind = (uint8_t)(((o.t[0] | o.t[1]) ? FOP_FLIP : 0) | ((o.a0 | o.a1) ? FOP_CNT : 0) |
                     (o.ph != NO_PH ? FOP_PH : 0) | (o.sbit != NO_SEL ? FOP_SEL : 0) |
                     ((o.c[1] | o.t[1] | (o.sbit != NO_SEL && o.sbit >= 64)) ? FOP_HI : 0));
}

struct PhasePair { double re0, im0, re1, im1; };   // phase for sel = 0, sel = 1

// ---- branching gate (Sec. 3.1, Eq. 2) ----------------------------------------
// For a label k with controls satisfied (and, for Givens, bit p != bit q) the
// pair is k0 = (x ? k ^ m : k), k1 = (x ? k : k ^ m) with x = bit sbit of k;
// k contributes M[0][x] a to k0 and M[1][x] a to k1. Otherwise k keeps a.
struct BranchOp {
  uint64_t c[2];        // controls
  uint64_t m[2];        // flip mask: one bit, or bits p and q for Givens
  uint32_t sbit;        // selector qubit (target, or p for Givens)
  uint32_t qbit;        // Givens: q; otherwise unused
  uint32_t givens;      // 1: also require bit p != bit q
  uint32_t real_m;      // 1: every entry of M is real
  double m_re[2][2];
  double m_im[2][2];
  // Pauli exponential exp(-i t/2 P) (pauli = 1): m = the X-or-Y mask of P, pz
  // its Z-or-Y mask, ny = (number of Y factors) mod 4, m_re diagonal = cos(t/2),
  // psin = sin(t/2); the off-diagonal entries depend on the pair (pauli_pair).
  uint64_t pz[2];
  uint32_t pauli;
  uint32_t ny;
  double psin;
};

// ---- bit-sliced form of a fused pass ------------------------------------------
// Labels of 32 entries are transposed into bit-planes (one 32-bit word per
// label bit, bit i = entry i). A gate then acts on 32 entries with a few logic
// ops: X with controls c is P[t] ^= AND(P[c]); pi/4 phases add a constant to a
// 3-plane counter; arbitrary phases record the planes on which they fire.
// A warp keeps a tile of G groups of 32 entries in shared memory, one row per
// plane and one column per group, and lane g walks the op list on column g.
// Rows: the label bits the pass needs (every valid bit of a 64-bit label half
// that the pass writes back, and the condition and selector bits elsewhere),
// then the aux rows (the counter's 3 planes, if any, then one fire plane per
// arbitrary phase slot), a scratch row for long condition lists and a row of
// all ones (unused condition slots read it, so a condition is always the AND
// of three rows). After the walk every entry gets its aux word back; its
// phase is the product over chunks of the aux bits of tables built on the
// device (fixed point, 2^62 = 1), one FP64 complex product per entry.
enum SOpKind : uint8_t { SOP_FLIP = 1, SOP_CNT = 2, SOP_FIRE = 4, SOP_SEL = 8, SOP_AND = 32 };
constexpr uint8_t kNoRow = 0xFF;

struct SOp {                // rows; the launch turns them into shared-memory offsets
  uint8_t kind;
  uint8_t c[3];             // condition rows (the ones row when unused)
  uint8_t t;                // flip row (SOP_AND: the row assigned)
  uint8_t s;                // selector row
  uint8_t f0, f1;           // aux rows written for sel = 0 / sel = 1 (f1 only with SEL)
  uint8_t a0, a1;           // counter steps for sel = 0 / 1 (mod 8)
};

constexpr uint32_t kMaxAuxBits = 64;     // counter (3) + fire slots
constexpr uint32_t kMaxFireSlots = kMaxAuxBits - 3;
constexpr uint32_t kBsMaxOps = 1024;     // op words of one bit-sliced launch (kernel parameters)
constexpr uint32_t kBsMaxChunkBits = 18; // aux bits per phase table (4 MiB)
constexpr uint64_t kBsJitMinNnz = 1ull << 20;   // SPS_OPT_BITSLICE_JIT = 1: from this bound
// Runs with at most this many aux bits get one table of every aux pattern's
// phase as doubles (2^bits x 16 B, 64 MiB at most): a lookup per entry and no
// product; more aux bits use fixed-point chunk tables and products.
constexpr uint32_t kBsDirectBits = 22;

struct BsPass {
  // the kernel compiled for this pass (sps_jit.cu), kept with the plan so a
  // reused plan launches it without generating its source again: the launch
  // form it was built for (jit_form, 0 = none), the kernel, its resident
  // blocks per SM at its shared memory
  mutable uint32_t jit_form = 0;
  mutable const void* jit_fn = nullptr;
  mutable int jit_bps = 0;
  // the same with a readout compiled in (jit_rd_key: the readout's form)
  mutable uint32_t jit_rd_form = 0;
  mutable std::string jit_rd_key;
  mutable const void* jit_rd_fn = nullptr;
  mutable int jit_rd_bps = 0;
  uint32_t nw = 0;            // 32-bit words of a label (nqubits / 32 rounded up)
  uint32_t nrows = 0;         // rows per tile column: label + aux + scratch + ones
  uint32_t label_rows = 0;
  uint32_t aux_row0 = 0, aux_bits = 0;
  uint32_t ones_row = 0;
  bool has_cnt = false;
  uint32_t word_bits[4] = {0, 0, 0, 0};  // bit j of word w has a row
  uint32_t word_out = 0;      // bit w: word w is written back
  uint8_t row_of[4][32];      // row of bit j of word w, or kNoRow
  std::vector<SOp> ops;
  std::vector<long long> factors;        // aux_bits x (re, im), fixed point 2^62
  uint32_t nchunks = 0;
  uint32_t chunk_shift[4] = {0, 0, 0, 0};
  uint32_t chunk_bits[4] = {0, 0, 0, 0};
  // 16-byte words of the launch's op stream: one per flip or scratch AND, two
  // per general op
  uint32_t op_words() const {
    uint32_t n = 0;
    for (const SOp& o : ops) n += (o.kind != SOP_FLIP && o.kind != SOP_AND) ? 2u : 1u;
    return n;
  }
  // An expansion from |0...0> fused in front of the run (build_bitslice_expand):
  // the launch generates the expansion's outputs instead of reading a state.
  // row_choice[r] = the choice bit (output index bit) that label row r holds,
  // -1 for a row of zeros; every label word is written; c_re, c_im = the
  // factor common to every output; ex_d = the expansion's gates.
  bool expand = false;
  std::vector<int8_t> row_choice;
  double c_re = 1.0, c_im = 0.0;
  uint32_t ex_d = 0;
  // aux_bits <= kBsDirectBits: the kernels look the phase up in one table of
  // 2^aux_bits doubles (re, im) built from the (two) fixed-point chunk tables
  bool direct = false;
  // 16-byte table entries: the fixed-point chunk tables, then the direct table
  uint64_t table_entries() const {
    return direct_offset() + (direct ? 1ull << aux_bits : 0ull);
  }
  uint64_t direct_offset() const {   // first entry of the direct table
    uint64_t t = 0;
    for (uint32_t c = 0; c < nchunks; ++c) t += 1ull << chunk_bits[c];
    return t;
  }
};

// ---- encoded op stream of a fused pass ------------------------------------------
// The direct and one-block fused passes walk the op list as a stream of 16-byte
// words. A header word {OPS_*, count, 0, 0} starts each run of ops of one form:
//   OPS_FLIP64   count words {c.lo, c.hi, t.lo, t.hi} (32-bit halves): a pure
//                flip whose condition and target lie in qubits 0..63;
//   OPS_FLIP128  count x 2 words: the 128-bit condition, then the target;
//   OPS_GEN      count x 3 words: FOp records (phases, counters, selectors),
//                except that the ph field holds the op's fire slots f0 | f1 << 8
//                (f1 for sel = 1, 0xFF if none): an arbitrary phase that applies
//                sets its slot bit, and the product of the phases of the set
//                bits is taken at the end from per-8-slot tables.
// A flip costs the walk one load and five logic instructions, a general op
// about four times that.
struct OpWord { uint32_t x, y, z, w; };
static_assert(sizeof(OpWord) == 16, "OpWord layout");
constexpr uint32_t OPS_FLIP64 = 1, OPS_FLIP128 = 2, OPS_GEN = 3;
struct Pass;
// Encodes the pass's ops (p.words) and builds its fire-slot tables (p.ftab).
void encode_ops(Pass* p);

// ---- a compiled pass -----------------------------------------------------------
enum PassKind : uint32_t { PASS_FUSED = 1, PASS_BRANCH = 2, PASS_EXPAND = 3, PASS_LAYER = 4 };

// Layer pass: up to kMaxLayerGates consecutive branching gates whose qubits
// (targets and controls) are pairwise disjoint, applied in one gather pass.
constexpr uint32_t kMaxLayerGates = 4;
// Most gates of one amplitude-only run (disjoint qubits; see launch_amp_part).
constexpr uint32_t kMaxAmpGates = 32;
// Most sign conditions of a sign-only phase run an attempt applies by parity.
constexpr uint32_t kMaxAmpParity = 64;

// Qubits known (on the host, conservatively) to hold one value in every stored
// label: bit q of known set => every label has bit q = bit q of val.
struct KnownBits {
  uint64_t known[2] = {0ull, 0ull};
  uint64_t val[2] = {0ull, 0ull};
};

// Expansion pass: d branching gates, each active on every entry and flipping
// only qubits known constant before it, so no two paths meet. Output (i, c)
// for c in [0, 2^d): label k_i ^ mask(c), amplitude a_i * factor(c), both taken
// from per-chunk tables over 8 gates (c = c0 | c1 << 8 | c2 << 16).
constexpr uint32_t kExpandChunk = 8;
constexpr uint32_t kMaxExpandGates = 24;

struct Pass {
  PassKind kind;
  uint64_t first_gate;
  uint32_t ngates = 0;      // fused: gates of the run (its ops may be fewer or more)
  // fused
  std::vector<FOp> ops;
  std::vector<OpWord> words;  // ops encoded for the direct walk (encode_ops)
  std::vector<double> ftab;   // fire-slot tables: chunks x 256 x (re, im) (encode_ops)
  std::vector<PhasePair> phases;
  bool has_perm = false;    // some op flips label bits
  bool has_phase = false;   // some op changes amplitudes
  uint32_t fire_slots = 0;  // aux bits its arbitrary phases need in bit-sliced form
  // branch
  BranchOp br{};
  uint64_t sup[2] = {0ull, 0ull};   // branch / layer: qubits its gates touch
  // layer
  std::vector<BranchOp> lay;        // its gates, in order
  std::vector<uint64_t> lay_gate;   // the index of each in the stream
  // expand
  std::vector<BranchOp> ex_ops; // its gates, in order
  std::vector<uint8_t> ex_x;    // value of each gate's selector qubit before it
  uint32_t ex_d = 0;            // gates
  bool ex_real = false;         // every path factor is real
  std::vector<double> ex_f;     // per chunk: 256 x (re, im) products of matrix entries
  std::vector<uint64_t> ex_m;   // per chunk: 256 x (lo, hi) xor of the flip masks
  uint32_t ex_chunks() const { return (ex_d + kExpandChunk - 1) / kExpandChunk; }
};

// One pass of a small-state run (k_small_run), stored in the plan arena.
struct RunPass {            // 64 bytes
  uint32_t kind;            // PASS_FUSED or PASS_BRANCH
  uint32_t nops;            // fused: gates of the run (the update count)
  uint32_t ops_off;         // byte offset of the encoded op stream in the arena
  uint32_t ph_off;          // fused: byte offset of the fire-slot tables
  uint32_t br_off;          // byte offset of the BranchOp
  uint32_t flags;           // bit 0: permutes, bit 1: changes amplitudes
  uint32_t pass_serial;     // small run: pass index in the apply + 1 (the launch adds
                            // its serial base); batch: pass index
  uint32_t nwords;          // fused: words of the encoded op stream
  uint64_t fail_tag;        // small run: first gate (the launch adds the apply serial)
  double eps2;
  double eps;
  uint64_t reserved2;
};
static_assert(sizeof(RunPass) == 64, "RunPass layout");

constexpr uint32_t kSmallCap = 2048;          // entries a small-state run holds
constexpr uint32_t kSmallThreads = 1024;
constexpr uint32_t kSmallTableSlots = 8192;   // input index table, load <= 25%

// Builds the bit-sliced form of a fused pass for an nqubits-qubit state.
void build_bitslice(const Pass& p, uint32_t nqubits, BsPass* out);
// The bit-sliced form of expansion pass `ex` (from |0...0>) followed by fused
// run `run`, as one pass: false unless every expansion gate flips one qubit
// and no output can be pruned at eps (every output factor's modulus above
// 2 eps).
bool build_bitslice_expand(const Pass& ex, const Pass& run, uint32_t nqubits, double eps,
                           BsPass* out);

// Bounds of one fused pass: ops, arbitrary phases (each a table entry of the
// bit-sliced form) and, below, its fire slots.
constexpr uint32_t kMaxFusedOps = 512;
constexpr uint32_t kMaxFusedPhases = 96;
constexpr uint32_t kDefaultMaxFusedOps = kMaxFusedOps;

// Validates and compiles; on a bad record returns SPS_ERR_ARG with *bad set.
// Gate commuting queues (Sec. 3.3): rewrites the stream so that H, Rx and Ry
// gates wait in per-qubit queues and cancel, merge or pass phase/permutation
// gates where a commutation identity allows; origin[i] is the input index of
// output gate i. Validates first (SPS_ERR_ARG with *bad).
sps_status commute_gates(const sps_gate* gates, size_t ngates, uint32_t nqubits,
                         std::vector<sps_gate>* out, std::vector<size_t>* origin, size_t* bad);

// With kb (nullable) the compiler tracks the known-constant qubits through the
// gates (updating *kb on success); if expand it forms expansion passes, if
// fold it resolves known qubits in fused runs (lower_known).
// layer_max > 1 groups consecutive disjoint branching gates into layer passes.
sps_status compile(const sps_gate* gates, size_t ngates, uint32_t nqubits,
                   uint32_t max_fused_ops, std::vector<Pass>* out, size_t* bad,
                   KnownBits* kb = nullptr, bool expand = false, bool fold = false,
                   uint32_t layer_max = 1);
// The most nonzeros a state can reach from |0...0> through the passes (every
// branching gate at most doubles the count), capped at the capacity.
uint64_t projected_peak(const std::vector<Pass>& passes, uint64_t capacity);

// ---- device-side control block -------------------------------------------------
constexpr int kMaskStripes = 32;
struct Ctl {
  unsigned long long nnz;        // entries in the current buffer
  unsigned long long out_count;  // compaction output counter of the running pass
  unsigned int cur;              // which of the two buffers holds the state
  unsigned int status;           // first device-side error (sps_status), 0 = none
  unsigned int fail_pass;        // pass serial of the failing pass
  unsigned int blocks_done;      // last-block detection in the compaction
  unsigned long long fail_gate;  // (apply serial << 32) | first gate of failing pass
  unsigned long long updates;    // sum over applied gates of the nonzeros before them
  // OR and AND of every stored label (qubits 0..63 in word 0): a qubit whose
  // OR and AND bits agree has the same value in every label. Three rotating
  // buffers: a pass that writes labels reads the masks of its input from
  // buffer rd, merges those of its output into buffer wr (fire-and-forget
  // atomics spread over kMaskStripes stripes, so blocks do not queue on one
  // address) and resets buffer rs for the pass after it; kernel boundaries
  // order the three. The host advances the rotation (MaskRing).
  unsigned long long lm[3][kMaskStripes][4];   // {or0, or1, and0, and1}
  // Amplitude-only branching passes: a pass whose gates meet only complete
  // groups and prune nothing keeps every label where it is, so it needs only
  // new amplitudes and an index of the labels that stays valid across such
  // passes.
  unsigned long long index_n;    // entries the index was built for (sets its size)
  unsigned int index_ok;         // the index table holds every label of the state
  unsigned int index_epoch;      // its epoch
  unsigned int amp_go;           // the running pass attempts the amplitude-only form
  unsigned int amp_state;        // 1: the amplitude-only form produced the pass's state
  unsigned int amp_fail;         // set by threads that find the form not applicable
  unsigned int amp_backoff;      // passes still to skip after failed attempts
  unsigned int amp_streak;       // failed attempts in a row
  // grid barrier of cooperative launches: generation << 16 | blocks arrived
  unsigned int grid_bar;
  // next chunk of 32 entries an amplitude-only attempt's warps take (zeroed
  // by the index launch before it and by the attempt's last block)
  unsigned long long chunk_next;
};

// Mask buffer indices of one label-writing launch, packed rd | wr << 8 | rs << 16.
struct MaskRing {
  uint32_t gen = 0;
  uint32_t reader() const { return gen % 3u; }
  uint32_t writer() {
    const uint32_t v = (gen % 3u) | (((gen + 1u) % 3u) << 8) | (((gen + 2u) % 3u) << 16);
    ++gen;
    return v;
  }
};
__host__ __device__ constexpr uint32_t mg_rd(uint32_t mg) { return mg & 0xFFu; }
__host__ __device__ constexpr uint32_t mg_wr(uint32_t mg) { return (mg >> 8) & 0xFFu; }
__host__ __device__ constexpr uint32_t mg_rs(uint32_t mg) { return (mg >> 16) & 0xFFu; }

struct SoA {
  uint64_t* lo;
  uint64_t* hi;   // unused (may be null) for 64-bit labels
  double* re;
  double* im;
};

struct Bufs { SoA b[2]; };

struct __align__(32) Slot {
  uint64_t lo, hi;
  double re, im;
};

constexpr uint64_t EMPTY = ~0ull;   // label bit 127 (or 63) is never set

// Table size for a branching pass with n_in input entries (both kernels of the
// pass compute it from the same n_in, so they agree without a host round trip).
__host__ __device__ inline uint32_t table_log2_for(unsigned long long n_in, uint32_t load_pct,
                                                   uint32_t max_log2) {
  const unsigned long long need = (2ull * n_in * 100ull + load_pct - 1) / load_pct;
  uint32_t lg = 8;
  while (lg < max_log2 && (1ull << lg) < need) ++lg;
  return lg;
}

// ---- kernel launchers (sps_kernels.cu) -----------------------------------------
struct LaunchCfg {
  int threads;
  int max_blocks;
  void* stream;
};

// All launchers return the number of kernels enqueued, or -1 on a launch error.
// `plog` (nullable) receives two words per launch for profiling: entries read
// and entries in the state afterwards.
int launch_table_clear(const LaunchCfg& lc, Slot* table, uint64_t nslots);
// words / ftab: the pass's encoded op stream and fire-slot tables in device memory
// lanes: labels per thread (1, 2, 4 or 8; 0 picks by the nonzero bound);
// fallback: 1 if an amplitude-only attempt before it may have taken the pass
int launch_fused(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, const Pass& p,
                 const OpWord* words, const double* ftab, uint64_t nnz_bound, uint32_t mg,
                 int lanes, uint32_t fallback, unsigned long long* plog);
struct BranchLaunch {
  BranchOp op;
  double eps;
  uint32_t load_pct, max_log2, probe_limit, pass_serial;
  int coop;
  uint64_t capacity, fail_tag;
  uint32_t mg;   // label-mask buffers (MaskRing): rd for the gather passes, all for the writer
  uint32_t fallback = 0;   // 1: runs only if the amplitude-only form did not take the pass
};
int launch_branch_emit(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, Slot* table,
                       const BranchLaunch& b, uint64_t nnz_bound, unsigned long long* plog);
int launch_branch_compact(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, Slot* table,
                          const BranchLaunch& b, uint64_t nnz_bound, unsigned long long* plog);
struct BsLaunch {
  const BsPass* plan;
  const long long* factors;  // device copy of plan->factors (plan arena)
  long long* tables;         // device table space (plan->table_entries() x 16 B)
  uint32_t build_tables;     // 1: build the tables from the factors first
  uint32_t ngates;           // gates of the run, for the update count
  uint32_t has_perm, has_phase;
  uint32_t groups;           // groups of 32 entries per warp tile (2..32), 0 = choose
  uint32_t mg;               // label-mask buffers (MaskRing)
  uint32_t fallback = 0;     // as in launch_fused
  // A probability readout summed by the expansion form as it stores (see
  // ReadoutFuse); nullptr: none. *rd_done is set to 1 if the launch sums it.
  const struct ReadoutFuse* rd = nullptr;
  uint32_t* rd_done = nullptr;
};
// sum |a|^2 over output labels k with (k & mask) == value, formed by a
// compiled expansion launch: per-block sums in part[0 .. cap), the total in *out
struct ReadoutFuse {
  uint64_t mask[2], value[2];
  double* part;
  double* out;
  uint32_t cap;
  uint32_t min_planes;   // summed only if it tests this many planes (or none can match)
};
// Returns the kernels enqueued (1 or more), 0 if the plan does not fit one
// launch (then the pass must take the direct form), -1 on a launch error.
int launch_fused_bs(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, const BsLaunch& b,
                    uint64_t nnz_bound, unsigned long long* plog);
// Builds the pass's phase tables from its factors (kernels enqueued, -1 on error).
int launch_bs_tables(const LaunchCfg& lc, const BsLaunch& b);
// The bit-sliced pass compiled for this plan (sps_jit.cu): the op walk as
// straight-line code on registers and every row offset a constant. Returns
// the kernels enqueued (tables included), 0 if this form is not available
// (runtime compiler missing or the compile failed: use launch_fused_bs), -1
// on a launch error.
int launch_fused_bs_jit(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, const BsLaunch& b,
                        uint64_t nnz_bound, unsigned long long* plog);
// Host-only check of the runtime compiler: generates and compiles the kernel
// of a small sample pass; returns 1 if it compiled, 0 if not available.
int bs_jit_selftest(char* log, size_t cap);
// Runs npasses consecutive passes (RunPass records at arena + pass_off) in one
// CTA with the state in shared memory; the host guarantees nnz <= kSmallCap.
int launch_small_run(void* stream, int key_words, Ctl* ctl, Bufs bufs, const unsigned char* arena,
                     uint32_t pass_off, uint32_t npasses, uint64_t capacity, uint32_t mg,
                     uint32_t serial_base, uint32_t apply_serial, unsigned long long* plog);
// Gather form of a branching pass (insert-once rule, Sec. 3.1) on the whole GPU:
// k_gather_build claims one slot per input label in an index table whose
// 64-bit slots hold (epoch << 32 | input index), so a new epoch per pass makes
// the table empty without clearing it; k_gather_emit looks up each active
// entry's partner, writes the pair once, prunes and compacts.
// part 0 launches k_gather_build, part 1 k_gather_emit.
int launch_gather_part(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs,
                       unsigned long long* itab, uint32_t epoch, const BranchLaunch& b,
                       uint64_t nnz_bound, int part, unsigned long long* plog);
int launch_itab_clear(const LaunchCfg& lc, unsigned long long* itab, uint64_t nslots);
// Layer pass (PASS_LAYER), gather form: part 0 indexes the labels that may be
// looked up, part 1 writes every group once (see sps_gather.cu).
struct LayerLaunch {
  BranchOp ops[kMaxLayerGates];
  uint32_t d;
  double eps;
  uint32_t load_pct, max_log2, pass_serial, mg;
  uint64_t capacity, fail_tag;
  uint32_t fallback;   // as in BranchLaunch
};
int launch_layer_part(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs,
                      unsigned long long* itab, uint32_t epoch, const LayerLaunch& l,
                      uint64_t nnz_bound, int part, unsigned long long* plog);
// Amplitude-only form of a run of branching passes: l.d gates (1..32) on
// pairwise disjoint qubits. part 0: unless an earlier failure says to skip
// this attempt, index every label (epoch `epoch`) if `force` or the device
// says the index is stale, and decide the attempt; part 1: the attempt
// itself, which produces the run's state only if every active group is
// complete (at most 16 members) and nothing is pruned (else the run's own
// passes, launched after it with fallback = 1, run).
struct AmpLaunch {
  BranchOp ops[kMaxAmpGates];
  uint32_t d;
  double eps;
  uint32_t load_pct, max_log2, pass_serial;
  uint64_t fail_tag;
  // optional phase-only fused run after the run (nwords == 0: none), walked on
  // every output before it is stored; fused_gates counts its gates
  const OpWord* words;
  const double* ftab;
  uint32_t nwords, fused_gates, has_phase;
  // or (npar > 0) a phase run of signs only: the amplitude is negated where an
  // odd number of the npar conditions (c0, c1 pairs: all bits set) hold
  uint64_t par[2 * kMaxAmpParity];
  uint32_t npar;
};
int launch_amp_part(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs,
                    unsigned long long* itab, uint32_t epoch, uint32_t force, const AmpLaunch& l,
                    uint64_t nnz_bound, int part, unsigned long long* plog);
// The passes of a run an amplitude-only attempt stands in for (its fallback),
// in one cooperative launch: at once done if the attempt took the run, else
// each pass as its separate kernels would run it, with grid barriers between
// them, then the phase-only run after them (a direct op stream, or a sign
// parity as the attempt applies it). Returns 1 when enqueued, 0 when the
// chain does not fit one launch (launch the passes one by one), -1 on a
// launch error.
constexpr uint32_t kChainSteps = kMaxAmpGates;
struct ChainStepDesc {
  uint32_t kind;    // PASS_BRANCH (gather form) or PASS_LAYER
  uint32_t epoch;   // its index-table epoch
  BranchLaunch br;  // PASS_BRANCH
  LayerLaunch lay;  // PASS_LAYER
};
struct ChainWalk {
  const OpWord* words;   // direct op stream (nwords > 0), or
  const double* ftab;
  uint32_t nwords, has_phase;
  const uint64_t* par;   // npar sign conditions (c0, c1 pairs)
  uint32_t npar;
  uint32_t ngates;       // gates of the run; 0: none after the passes
};
int launch_chain(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs,
                 unsigned long long* itab, const ChainStepDesc* steps, uint32_t nsteps,
                 const ChainWalk& w, uint64_t nnz_bound, unsigned long long* plog);
// Runs the grid barrier of k_chain on a scratch control block (8 blocks, three
// barriers; block skip_block misses the first); *status receives the block's
// status word. Returns 0, or -1 on a CUDA error.
int barrier_selftest(uint32_t skip_block, uint32_t spins, int* status);
// Expansion pass (PASS_EXPAND); f, m: its tables in device memory.
struct ExpandLaunch {
  const double* f;
  const uint64_t* m;
  uint32_t d, real, pass_serial, mg;
  double eps;
  uint64_t capacity, fail_tag;
  // optional fused run applied to the outputs before they are stored
  // (nwords == 0: none); fused_gates counts its gates for the update count
  const OpWord* words;
  const double* ftab;
  uint32_t nwords, fused_gates, has_phase;
  // 1: the input is |0...0> (a reset not yet enqueued): the kernel does the
  // reset's work on the control block and reads no entry
  uint32_t from_reset;
};
int launch_expand(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, const ExpandLaunch& e,
                  uint64_t nnz_bound, unsigned long long* plog);
// Measurement with collapse: partials holds 2 * nblocks doubles; res receives
// {outcome, probability of the outcome, 1 / sqrt(p_outcome)}.
int launch_measure(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs, uint32_t qubit,
                   double r, double* partials, int nblocks, double* res, uint64_t nnz_bound,
                   uint32_t mg, unsigned long long* plog);
int launch_probability(const LaunchCfg& lc, int key_words, Ctl* ctl, Bufs bufs,
                       uint64_t mask_lo, uint64_t mask_hi, uint64_t val_lo, uint64_t val_hi,
                       double* partials, int nblocks, double* result,
                       unsigned long long* plog = nullptr);
// mg: label-mask buffers of a launch that writes labels (MaskRing::writer)
int launch_set_nnz(void* stream, Ctl* ctl, unsigned long long nnz, uint32_t mg);
int launch_reset_state(void* stream, int key_words, Ctl* ctl, Bufs bufs, uint32_t mg);
// mg != kNoMasks: also merge the OR/AND masks of the checked labels
constexpr uint32_t kNoMasks = 0xFFFFFFFFu;
int launch_check_labels(void* stream, int key_words, Ctl* ctl, Bufs bufs,
                        uint64_t lim_lo, uint64_t lim_hi, unsigned int* bad_flag, uint64_t n,
                        uint32_t mg);
int launch_reset_status(void* stream, Ctl* ctl);

}  // namespace sps
