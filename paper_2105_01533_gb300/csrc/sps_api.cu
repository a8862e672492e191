// C ABI of libsps (see include/sps.h). Host orchestration only: validation,
// compilation into passes, buffer management and kernel enqueue. Every step of
// the gate application runs in the kernels of sps_kernels.cu.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <memory>
#include <vector>

#include "sps.h"
#include "sps_batch.h"
#include "sps_internal.h"

using namespace sps;

namespace {

std::mutex g_alloc_mu;
sps_alloc_fn g_alloc = nullptr;
sps_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

constexpr size_t kProfileCap = 1 << 16;   // profiled launches kept between reads

struct Allocation {
  void* ptr;
  size_t bytes;
};

// A compiled apply: its passes, how they are launched and the arena image
// they read. A state keeps the last one: an apply with the same gates, prune
// threshold, options, starting knowledge and nonzero bound reuses it, and its
// image while the arena still holds it, instead of compiling and uploading.
struct ApplyPlan {
  std::vector<sps_gate> gates;
  uint64_t eps_bits = 0;
  KnownBits kb_in, kb_out;
  uint64_t bound_in = 0;
  std::vector<uint64_t> opts;
  std::vector<Pass> passes;
  std::vector<size_t> seg_end;      // > 0: a small-state run starts here, ends there
  std::vector<uint64_t> bound_at;   // nonzero bound before each pass
  std::vector<BsPass> bs;           // bit-sliced plans of long fused runs
  std::vector<size_t> bs_off;       // their phase factors in the arena image
  std::vector<uint64_t> bs_tab;     // their phase tables: first entry in the table space
  uint64_t bs_tab_entries = 0;      // table space the plan needs (16 B per entry)
  // passes 0 and 1 as one compiled launch when pass 0 is an expansion from a
  // pending reset and pass 1 a bit-sliced run (build_bitslice_expand)
  BsPass bs_ex;
  bool bs_ex_ok = false;
  size_t bs_ex_off = 0;             // its factors in the arena image
  uint64_t bs_ex_tab = 0;           // its phase tables in the table space
  std::vector<size_t> run_off;      // small run: its RunPass array; direct fused pass: its
                                    // op stream; expansion: its factor tables
  std::vector<size_t> ph_off;       // direct fused pass: its fire-slot tables; expansion:
                                    // its mask tables
  std::vector<uint8_t> walk_next;   // expansion: the fused pass after it runs in its kernel
  std::vector<size_t> amp_end;      // > 0: a run of branching passes on disjoint qubits starts
                                    // here (ends there) with one amplitude-only attempt
  std::vector<uint8_t> amp_walk;    // run start: the phase-only fused pass after the run is
                                    // walked by the attempt (and is its fallback)
  std::vector<std::vector<uint64_t>> amp_par;   // run start: that pass as sign conditions
                                                // (c0, c1 pairs) when it holds only signs
  std::vector<unsigned char> image;
};

}  // namespace

struct sps_state {
  uint32_t nqubits = 0;
  int kw = 1;                 // label words: 1 (<= 63 qubits) or 2
  uint64_t capacity = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 0;
  // memory
  sps_alloc_fn alloc = nullptr;
  sps_free_fn release = nullptr;
  void* alloc_ctx = nullptr;
  std::vector<Allocation> allocs;
  Ctl* ctl = nullptr;
  Ctl* ctl_host = nullptr;    // pinned mirror
  Bufs bufs{};
  Slot* table = nullptr;            // scatter-form table, allocated on first use
  uint32_t max_log2 = 8;
  uint64_t table_slots = 0;
  unsigned long long* itab = nullptr;  // gather-form index table
  uint32_t itab_log2 = 8;
  uint32_t epoch = 0;
  MaskRing masks;             // rotation of the device label-mask buffers
  std::unique_ptr<ApplyPlan> plan;   // the last compiled apply
  bool plan_resident = false;        // the arena holds plan->image
  KnownBits kb;               // qubits known constant once every enqueued pass ran
  bool expand = true;         // SPS_OPT_EXPAND
  bool fold = true;           // SPS_OPT_FOLD
  bool commute = false;       // SPS_OPT_COMMUTE
  uint32_t layer_max = kMaxLayerGates;   // SPS_OPT_LAYER_GATES
  bool expand_walk = true;               // SPS_OPT_EXPAND_WALK
  int fused_labels = 0;                  // SPS_OPT_FUSED_LABELS (0: by size)
  bool amp = true;                       // SPS_OPT_AMP_ONLY
  bool amp_force = true;                 // the label index must be rebuilt before use
  bool reset_pending = false;            // sps_reset not yet enqueued (see flush_reset)
  int branch_form = 0;               // 0 auto (gather), 1 scatter, 2 gather
  double* partials = nullptr;
  double* dresult = nullptr;
  double* dmeasure = nullptr;   // {outcome, probability, scale} of the last measurement
  double* hresult = nullptr;  // pinned
  unsigned* dflag = nullptr;
  unsigned* hflag = nullptr;  // pinned
  int prob_blocks = 0;
  // a registered readout (sps_set_readout): summed by a compiled expansion
  // launch that ends an sps_apply; valid while version == rd_version
  bool rd_on = false;
  uint64_t rd_mask[2] = {0ull, 0ull}, rd_value[2] = {0ull, 0ull};
  double* rd_buf = nullptr;    // rd_cap block sums, then the sum
  uint32_t rd_cap = 0;
  uint64_t version = 1;        // bumped by every call that changes the state
  uint64_t rd_version = 0;     // version whose readout sum is in rd_buf[rd_cap]
  // options
  uint32_t load_pct = 50;
  uint32_t probe_limit = 0;   // 0 = table size
  int threads = 256;
  uint32_t max_fused_ops = kDefaultMaxFusedOps;
  int coop = 1;
  uint32_t bitslice_min_ops = 8;
  uint64_t bitslice_min_nnz = 1u << 18;   // below this the direct kernel is faster
  uint32_t bs_groups = 0;                  // bit-sliced tile groups, 0 = heuristic
  int bs_jit = 1;                          // SPS_OPT_BITSLICE_JIT
  bool plan_cache = true;                  // SPS_OPT_PLAN_CACHE
  bool chain = true;                       // SPS_OPT_FALLBACK_CHAIN
  uint32_t rd_min_planes = 8;              // SPS_OPT_READOUT_MIN_PLANES
  uint32_t small_cap = kSmallCap;   // 0 disables small-state runs
  // plan arena: op streams, factors and tables of the current sps_apply
  unsigned char* arena = nullptr;
  size_t arena_cap = 0;
  // phase tables of the bit-sliced passes, built on the device when the plan
  // is uploaded
  long long* bs_tables = nullptr;
  size_t bs_tables_cap = 0;
  struct Staging {
    unsigned char* host = nullptr;   // pinned
    size_t cap = 0;
    cudaEvent_t copied = nullptr;    // recorded after the copy out of `host`
    bool pending = false;
  };
  Staging staging[4];
  unsigned staging_next = 0;
  // profiling (SPS_OPT_PROFILE)
  bool profile = false;
  unsigned long long* dlog = nullptr;      // 2 words per profiled launch
  unsigned long long* hlog = nullptr;      // pinned copy
  struct Pending {
    cudaEvent_t start, stop;
    uint32_t kind, pass_serial, nops, flags;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  // bookkeeping
  uint64_t nnz_bound = 1;
  uint32_t pass_serial = 0;
  uint32_t apply_serial = 0;
  sps_counters counters{};
};

namespace {

void* default_alloc(void*, size_t bytes, void* stream) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void default_free(void*, void* p, size_t, void* stream) {
  cudaFreeAsync(p, (cudaStream_t)stream);
}

sps_status dev_alloc(sps_state* s, size_t bytes, void** out) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = s->alloc(s->alloc_ctx, bytes, s->stream);
  if (!p) return SPS_ERR_OOM;
  s->allocs.push_back({p, bytes});
  *out = p;
  return SPS_OK;
}

void release_all(sps_state* s) {
  cudaStreamSynchronize(s->stream);
  for (auto& a : s->allocs) s->release(s->alloc_ctx, a.ptr, a.bytes, s->stream);
  s->allocs.clear();
  cudaStreamSynchronize(s->stream);
  if (s->ctl_host) cudaFreeHost(s->ctl_host);
  if (s->hresult) cudaFreeHost(s->hresult);
  if (s->hflag) cudaFreeHost(s->hflag);
  if (s->hlog) cudaFreeHost(s->hlog);
  s->hlog = nullptr;
  for (auto& p : s->pending) {
    cudaEventDestroy(p.start);
    cudaEventDestroy(p.stop);
  }
  s->pending.clear();
  for (auto e : s->event_pool) cudaEventDestroy(e);
  s->event_pool.clear();
  for (auto& st : s->staging) {
    if (st.host) cudaFreeHost(st.host);
    if (st.copied) cudaEventDestroy(st.copied);
    st = sps_state::Staging();
  }
  s->ctl_host = nullptr;
  s->hresult = nullptr;
  s->hflag = nullptr;
  cudaGetLastError();
}

}  // namespace

void* sps::hook_alloc(size_t bytes, void* stream) {
  sps_alloc_fn a;
  sps_free_fn f;
  void* ctx;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc ? g_alloc : default_alloc;
    f = g_alloc ? g_free : default_free;
    ctx = g_alloc ? g_alloc_ctx : nullptr;
  }
  const size_t rounded = (bytes + 255) & ~size_t(255);
  void* p = a(ctx, rounded, stream);
  // the kernels' vector loads rely on the alignment the hook promises
  if (p && (reinterpret_cast<uintptr_t>(p) & 255u) != 0u) {
    f(ctx, p, rounded, stream);
    return nullptr;
  }
  return p;
}

void sps::hook_free(void* p, size_t bytes, void* stream) {
  sps_free_fn f;
  void* ctx;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    f = g_alloc ? g_free : default_free;
    ctx = g_alloc ? g_alloc_ctx : nullptr;
  }
  f(ctx, p, (bytes + 255) & ~size_t(255), stream);
}

namespace {

LaunchCfg cfg_of(const sps_state* s) {
  LaunchCfg lc;
  lc.threads = s->threads;
  lc.max_blocks = s->sms * (2048 / s->threads);
  lc.stream = s->stream;
  return lc;
}

sps_status cuda_ok(cudaError_t e) {
  if (e == cudaSuccess) return SPS_OK;
  cudaGetLastError();
  return SPS_ERR_CUDA;
}

// Reads the control block after the stream drains.
// sps_reset only records the reset: the next apply that starts with an
// expansion pass builds its outputs from |0...0> itself (one launch fewer per
// reset-apply cycle); any other use of the state enqueues the reset first.
sps_status flush_reset(sps_state* s) {
  if (!s->reset_pending) return SPS_OK;
  s->reset_pending = false;
  if (launch_reset_state(s->stream, s->kw, s->ctl, s->bufs, s->masks.writer()) < 0)
    return cuda_ok(cudaGetLastError());
  s->counters.kernel_launches += 1;
  return SPS_OK;
}

sps_status read_ctl(sps_state* s) {
  const sps_status fs = flush_reset(s);
  if (fs != SPS_OK) return fs;
  if (cudaMemcpyAsync(s->ctl_host, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream) !=
      cudaSuccess)
    return cuda_ok(cudaGetLastError());
  return cuda_ok(cudaStreamSynchronize(s->stream));
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void label_limits(uint32_t nq, uint64_t* lim0, uint64_t* lim1) {
  *lim0 = nq >= 64 ? ~0ull : ((1ull << nq) - 1);
  *lim1 = nq <= 64 ? 0ull : (nq >= 128 ? ~0ull : ((1ull << (nq - 64)) - 1));
}

// The state is |0...0>: every qubit known, value 0.
void know_all_zero(sps_state* s) {
  label_limits(s->nqubits, &s->kb.known[0], &s->kb.known[1]);
  s->kb.val[0] = s->kb.val[1] = 0ull;
}

// After a failure nothing is assumed.
void know_nothing(sps_state* s) {
  s->kb = KnownBits();
  s->amp_force = true;
}

// Knowledge from the label masks the device holds for the current state
// (stream synchronised): a qubit is known where OR and AND agree.
sps_status know_from_device(sps_state* s) {
  unsigned long long lm[kMaskStripes][4];
  if (cudaMemcpy(lm, s->ctl->lm[s->masks.reader()], sizeof(lm), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return cuda_ok(cudaGetLastError());
  uint64_t o0 = 0, o1 = 0, a0 = ~0ull, a1 = ~0ull;
  for (int i = 0; i < kMaskStripes; ++i) {
    o0 |= lm[i][0];
    o1 |= lm[i][1];
    a0 &= lm[i][2];
    a1 &= lm[i][3];
  }
  uint64_t lim0, lim1;
  label_limits(s->nqubits, &lim0, &lim1);
  s->kb.known[0] = ~(o0 ^ a0) & lim0;
  s->kb.known[1] = ~(o1 ^ a1) & lim1;
  s->kb.val[0] = o0 & s->kb.known[0];
  s->kb.val[1] = o1 & s->kb.known[1];
  return SPS_OK;
}

cudaEvent_t take_event(sps_state* s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Makes the device plan arena at least `bytes` long. The old arena is released
// in stream order, after the kernels already enqueued that read it.
sps_status ensure_arena(sps_state* s, size_t bytes) {
  if (bytes <= s->arena_cap) return SPS_OK;
  size_t cap = s->arena_cap ? s->arena_cap : (1u << 20);
  while (cap < bytes) cap *= 2;
  void* p = s->alloc(s->alloc_ctx, cap, s->stream);
  if (!p) return SPS_ERR_OOM;
  if (s->arena) {
    for (auto it = s->allocs.begin(); it != s->allocs.end(); ++it) {
      if (it->ptr == s->arena) {
        s->release(s->alloc_ctx, it->ptr, it->bytes, s->stream);
        s->allocs.erase(it);
        break;
      }
    }
  }
  s->allocs.push_back({p, cap});
  s->arena = (unsigned char*)p;
  s->arena_cap = cap;
  return SPS_OK;
}

// Makes the bit-sliced phase-table space at least `bytes` long (the old one is
// released in stream order, like the arena).
sps_status ensure_bs_tables(sps_state* s, size_t bytes) {
  if (bytes <= s->bs_tables_cap) return SPS_OK;
  size_t cap = s->bs_tables_cap ? s->bs_tables_cap : (1u << 20);
  while (cap < bytes) cap *= 2;
  void* p = s->alloc(s->alloc_ctx, cap, s->stream);
  if (!p) return SPS_ERR_OOM;
  if (s->bs_tables) {
    for (auto it = s->allocs.begin(); it != s->allocs.end(); ++it) {
      if (it->ptr == s->bs_tables) {
        s->release(s->alloc_ctx, it->ptr, it->bytes, s->stream);
        s->allocs.erase(it);
        break;
      }
    }
  }
  s->allocs.push_back({p, cap});
  s->bs_tables = (long long*)p;
  s->bs_tables_cap = cap;
  return SPS_OK;
}

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// The scatter-form table (32-byte slots for 2 * capacity labels at 50% load)
// is large, so it is only allocated when that form is first used.
sps_status ensure_scatter_table(sps_state* s) {
  if (s->table) return SPS_OK;
  void* p = nullptr;
  const sps_status st = dev_alloc(s, s->table_slots * sizeof(Slot), &p);
  if (st != SPS_OK) return st;
  s->table = (Slot*)p;
  if (launch_table_clear(cfg_of(s), s->table, s->table_slots) < 0) return cuda_ok(cudaGetLastError());
  s->counters.kernel_launches += 1;
  return SPS_OK;
}

// Next pinned staging buffer of at least `bytes`; waits only if the copy that
// last used it has not finished (the ring lets the host run ahead of the GPU).
sps_status take_staging(sps_state* s, size_t bytes, sps_state::Staging** out) {
  sps_state::Staging& st = s->staging[s->staging_next];
  s->staging_next = (s->staging_next + 1) % 4;
  if (st.pending) {
    if (cudaEventSynchronize(st.copied) != cudaSuccess) return cuda_ok(cudaGetLastError());
    st.pending = false;
  }
  if (!st.copied && cudaEventCreateWithFlags(&st.copied, cudaEventDisableTiming) != cudaSuccess)
    return cuda_ok(cudaGetLastError());
  if (st.cap < bytes) {
    if (st.host) cudaFreeHost(st.host);
    st.host = nullptr;
    st.cap = 0;
    size_t cap = 1u << 16;
    while (cap < bytes) cap *= 2;
    if (cudaMallocHost((void**)&st.host, cap) != cudaSuccess) {
      cudaGetLastError();
      return SPS_ERR_OOM;
    }
    st.cap = cap;
  }
  *out = &st;
  return SPS_OK;
}

// Brackets one launch with events when profiling; returns the log slot or null.
struct ProfScope {
  sps_state* s;
  sps_state::Pending rec{};
  unsigned long long* slot = nullptr;
  bool on = false;
  ProfScope(sps_state* st, uint32_t kind, uint32_t serial, uint32_t nops, uint32_t flags) : s(st) {
    if (!s->profile || s->pending.size() >= kProfileCap) return;
    rec.start = take_event(s);
    rec.stop = take_event(s);
    if (!rec.start || !rec.stop) return;
    rec.kind = kind;
    rec.pass_serial = serial;
    rec.nops = nops;
    rec.flags = flags;
    slot = s->dlog + 2 * s->pending.size();
    on = cudaEventRecord(rec.start, s->stream) == cudaSuccess;
  }
  void done() {
    if (!on) return;
    if (cudaEventRecord(rec.stop, s->stream) == cudaSuccess) s->pending.push_back(rec);
  }
};

}  // namespace

extern "C" {

int sps_jit_selftest(char* log, size_t cap) { return bs_jit_selftest(log, cap); }

const char* sps_status_str(sps_status st) {
  switch (st) {
    case SPS_OK: return "ok";
    case SPS_ERR_ARG: return "invalid argument";
    case SPS_ERR_CAPACITY: return "capacity exceeded";
    case SPS_ERR_TABLE_FULL: return "hash table probe limit reached";
    case SPS_ERR_CUDA: return "CUDA error";
    case SPS_ERR_OOM: return "out of device memory";
    case SPS_ERR_NO_DEVICE: return "no CUDA device";
    case SPS_ERR_TIMEOUT: return "device-side wait timed out";
  }
  return "unknown status";
}

sps_status sps_set_allocator(sps_alloc_fn alloc, sps_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return SPS_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = release;
  g_alloc_ctx = ctx;
  return SPS_OK;
}

sps_status sps_create(uint32_t nqubits, uint64_t capacity, void* cuda_stream, sps_state** out) {
  if (!out) return SPS_ERR_ARG;
  *out = nullptr;
  if (nqubits < 1 || nqubits > 127 || capacity < 1 || capacity > (1ull << 34)) return SPS_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return SPS_ERR_NO_DEVICE;
  }
  sps_state* s = new (std::nothrow) sps_state;
  if (!s) return SPS_ERR_OOM;
  s->nqubits = nqubits;
  s->kw = nqubits <= 63 ? 1 : 2;
  s->capacity = capacity;
  s->stream = (cudaStream_t)cuda_stream;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    s->alloc = g_alloc ? g_alloc : default_alloc;
    s->release = g_alloc ? g_free : default_free;
    s->alloc_ctx = g_alloc ? g_alloc_ctx : nullptr;
  }
  sps_status st = SPS_OK;
  auto fail = [&](sps_status e) {
    release_all(s);
    delete s;
    return e;
  };
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(SPS_ERR_CUDA);
  }
  // table: 2 * capacity labels at the default 50% load, power of two
  s->max_log2 = table_log2_for(capacity, 50, 40);
  s->table_slots = 1ull << s->max_log2;
  s->prob_blocks = s->sms * 4 < 2048 ? s->sms * 4 : 2048;   // all resident
  void* p = nullptr;
  for (int b = 0; b < 2; ++b) {
    if ((st = dev_alloc(s, capacity * 8, &p)) != SPS_OK) return fail(st);
    s->bufs.b[b].lo = (uint64_t*)p;
    if (s->kw == 2) {
      if ((st = dev_alloc(s, capacity * 8, &p)) != SPS_OK) return fail(st);
      s->bufs.b[b].hi = (uint64_t*)p;
    }
    if ((st = dev_alloc(s, capacity * 8, &p)) != SPS_OK) return fail(st);
    s->bufs.b[b].re = (double*)p;
    if ((st = dev_alloc(s, capacity * 8, &p)) != SPS_OK) return fail(st);
    s->bufs.b[b].im = (double*)p;
  }
  s->itab_log2 = table_log2_for((capacity + 1) / 2, 50, 40);
  if ((st = dev_alloc(s, (sizeof(unsigned long long) << s->itab_log2), &p)) != SPS_OK) return fail(st);
  s->itab = (unsigned long long*)p;
  if ((st = dev_alloc(s, sizeof(Ctl), &p)) != SPS_OK) return fail(st);
  s->ctl = (Ctl*)p;
  // partials: 2 per block (the measurement's two sums), then the probability
  // result and the measurement's three results
  if ((st = dev_alloc(s, sizeof(double) * (2 * s->prob_blocks + 4), &p)) != SPS_OK) return fail(st);
  s->partials = (double*)p;
  s->dresult = s->partials + 2 * s->prob_blocks;
  s->dmeasure = s->dresult + 1;
  if ((st = dev_alloc(s, 256, &p)) != SPS_OK) return fail(st);
  s->dflag = (unsigned*)p;
  if ((st = dev_alloc(s, 2 * sizeof(unsigned long long) * kProfileCap, &p)) != SPS_OK) return fail(st);
  s->dlog = (unsigned long long*)p;
  if (cudaMallocHost((void**)&s->ctl_host, sizeof(Ctl)) != cudaSuccess ||
      cudaMallocHost((void**)&s->hresult, sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&s->hflag, sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost((void**)&s->hlog, 2 * sizeof(unsigned long long) * kProfileCap) != cudaSuccess) {
    cudaGetLastError();
    return fail(SPS_ERR_OOM);
  }
  // |0...0>: one entry (label 0, amplitude 1)
  static const double kOne = 1.0;
  SoA b0 = s->bufs.b[0];
  bool ok = cudaMemsetAsync(b0.lo, 0, 8, s->stream) == cudaSuccess &&
            (s->kw == 1 || cudaMemsetAsync(b0.hi, 0, 8, s->stream) == cudaSuccess) &&
            cudaMemcpyAsync(b0.re, &kOne, 8, cudaMemcpyHostToDevice, s->stream) == cudaSuccess &&
            cudaMemsetAsync(b0.im, 0, 8, s->stream) == cudaSuccess &&
            cudaMemsetAsync(s->ctl, 0, sizeof(Ctl), s->stream) == cudaSuccess;
  if (!ok) return fail(SPS_ERR_CUDA);
  LaunchCfg lc = cfg_of(s);
  if (launch_itab_clear(lc, s->itab, 1ull << s->itab_log2) < 0 ||
      launch_reset_state(s->stream, s->kw, s->ctl, s->bufs, s->masks.writer()) < 0)
    return fail(SPS_ERR_CUDA);
  s->counters.kernel_launches += 2;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return fail(cuda_ok(cudaGetLastError()));
  s->nnz_bound = 1;
  know_all_zero(s);
  *out = s;
  return SPS_OK;
}

sps_status sps_reset(sps_state* s) {
  if (!s) return SPS_ERR_ARG;
  ++s->version;
  s->amp_force = true;
  s->reset_pending = true;   // enqueued by the next use of the state (flush_reset)
  s->nnz_bound = 1;
  know_all_zero(s);
  return SPS_OK;
}

sps_status sps_profile_read(sps_state* s, sps_kernel_record* out, size_t cap, size_t* n) {
  if (!s || !n || (cap && !out)) return SPS_ERR_ARG;
  sps_status st = cuda_ok(cudaStreamSynchronize(s->stream));
  if (st != SPS_OK) return st;
  const size_t have = s->pending.size();
  if (have &&
      cudaMemcpy(s->hlog, s->dlog, 2 * sizeof(unsigned long long) * have, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return cuda_ok(cudaGetLastError());
  const size_t take = have < cap ? have : cap;
  for (size_t i = 0; i < take; ++i) {
    const auto& p = s->pending[i];
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.start, p.stop) != cudaSuccess) {
      cudaGetLastError();
      ms = -1.0f;
    }
    out[i].kind = p.kind;
    out[i].pass_serial = p.pass_serial;
    out[i].ms = ms;
    out[i].nops = p.nops;
    out[i].n_in = s->hlog[2 * i];
    out[i].n_out = s->hlog[2 * i + 1];
    out[i].flags = p.flags;
    out[i].label_bytes = 8u * (uint32_t)s->kw;
    s->event_pool.push_back(p.start);
    s->event_pool.push_back(p.stop);
  }
  // keep the rest queued, with their log words moved to the front
  if (take < have) {
    const size_t rest = have - take;
    if (cudaMemcpy(s->dlog, s->hlog + 2 * take, 2 * sizeof(unsigned long long) * rest,
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return cuda_ok(cudaGetLastError());
  }
  s->pending.erase(s->pending.begin(), s->pending.begin() + take);
  *n = take;
  return SPS_OK;
}

void sps_destroy(sps_state* s) {
  if (!s) return;
  release_all(s);
  delete s;
}

// Upper bound on the nonzeros after pass p, given bound b before it.
static uint64_t bound_after(const Pass& p, uint64_t b, uint64_t capacity) {
  uint32_t doublings = 0;
  if (p.kind == PASS_BRANCH) doublings = 1;
  if (p.kind == PASS_EXPAND) doublings = p.ex_d;
  if (p.kind == PASS_LAYER) doublings = (uint32_t)p.lay.size();
  for (uint32_t k = 0; k < doublings && b < capacity; ++k) b *= 2;
  return b < capacity ? b : capacity;
}

// A fresh 16-bit epoch for the index table; when it wraps, every slot is made
// free again (which also drops the label index of amplitude-only passes).
static sps_status next_epoch(sps_state* s, const LaunchCfg& lc) {
  if (++s->epoch == 0x10000u) {
    if (launch_itab_clear(lc, s->itab, 1ull << s->itab_log2) < 0) return cuda_ok(cudaGetLastError());
    s->counters.kernel_launches += 1;
    s->epoch = 1;
    s->amp_force = true;
  }
  return SPS_OK;
}

// The amplitude-only attempt of a run of gather-form branching passes, d gates
// in all (index check or rebuild, then the attempt); the run's own kernels,
// launched after it with fallback = 1, run only if it did not take the run.
static sps_status launch_amp_attempt(sps_state* s, const LaunchCfg& lc, const BranchOp* ops,
                                     uint32_t d, double prune_eps, uint32_t serial, uint64_t tag,
                                     const Pass* walk, const OpWord* words, const double* ftab,
                                     const std::vector<uint64_t>* par) {
  const sps_status es = next_epoch(s, lc);
  if (es != SPS_OK) return es;
  AmpLaunch l;
  std::memset(&l, 0, sizeof(l));
  l.d = d;
  for (uint32_t j = 0; j < d; ++j) l.ops[j] = ops[j];
  l.eps = prune_eps;
  l.load_pct = s->load_pct;
  l.max_log2 = s->itab_log2;
  l.pass_serial = serial;
  l.fail_tag = tag;
  if (walk && par) {   // the sign-only run after the run, as a parity
    l.fused_gates = walk->ngates;
    l.npar = (uint32_t)(par->size() / 2);
    for (size_t c = 0; c < par->size(); ++c) l.par[c] = (*par)[c];
  } else if (walk) {   // the phase-only run after the run, walked on the outputs
    l.words = words;
    l.ftab = ftab;
    l.nwords = (uint32_t)walk->words.size();
    l.fused_gates = walk->ngates;
    l.has_phase = walk->has_phase ? 1u : 0u;
  }
  const uint32_t force = s->amp_force ? 1u : 0u;
  {
    ProfScope pi(s, 9, serial, d, 0u);
    const int n = launch_amp_part(lc, s->kw, s->ctl, s->bufs, s->itab, s->epoch, force, l,
                                  s->nnz_bound, 0, pi.slot);
    pi.done();
    if (n < 0) return cuda_ok(cudaGetLastError());
  }
  {
    ProfScope pa(s, 10, serial, d, walk ? 6u : 2u);
    const int n = launch_amp_part(lc, s->kw, s->ctl, s->bufs, s->itab, s->epoch, force, l,
                                  s->nnz_bound, 1, pa.slot);
    pa.done();
    if (n < 0) return cuda_ok(cudaGetLastError());
  }
  s->amp_force = false;
  s->counters.kernel_launches += 2;
  return SPS_OK;
}

// One branching pass on the whole GPU (gather form, or scatter form when chosen
// or when the capacity needs 64-bit table indices); advances the nonzero bound.
// fallback: the gather kernels run only if an amplitude-only attempt launched
// just before did not take the pass.
static sps_status launch_branch_pass(sps_state* s, const LaunchCfg& lc, const BranchOp& op,
                                     double prune_eps, uint32_t serial, uint64_t tag,
                                     uint32_t limit, uint32_t fallback = 0) {
  BranchLaunch b;
  b.op = op;
  b.eps = prune_eps;
  b.load_pct = s->load_pct;
  b.max_log2 = s->max_log2;
  b.probe_limit = limit;
  b.pass_serial = serial;
  b.coop = s->coop;
  b.capacity = s->capacity;
  b.fail_tag = tag;
  b.mg = s->masks.writer();   // the pass writes labels: compaction or gather emit
  b.fallback = fallback;
  const bool scatter = s->branch_form == 1 || s->capacity >= (1ull << 32);
  if (scatter) {
    const sps_status ts = ensure_scatter_table(s);
    if (ts != SPS_OK) return ts;
    {
      ProfScope ps(s, 2, serial, 1, 3u);
      const int n = launch_branch_emit(lc, s->kw, s->ctl, s->bufs, s->table, b, s->nnz_bound, ps.slot);
      ps.done();
      if (n < 0) return cuda_ok(cudaGetLastError());
    }
    {
      ProfScope ps(s, 3, serial, 1, 3u);
      const int n = launch_branch_compact(lc, s->kw, s->ctl, s->bufs, s->table, b, s->nnz_bound, ps.slot);
      ps.done();
      if (n < 0) return cuda_ok(cudaGetLastError());
    }
  } else {
    const sps_status es = next_epoch(s, lc);
    if (es != SPS_OK) return es;
    b.max_log2 = s->itab_log2;
    ProfScope pb(s, 5, serial, 1, 3u);
    int n = launch_gather_part(lc, s->kw, s->ctl, s->bufs, s->itab, s->epoch, b, s->nnz_bound, 0, pb.slot);
    pb.done();
    if (n < 0) return cuda_ok(cudaGetLastError());
    ProfScope pe(s, 6, serial, 1, 3u);
    n = launch_gather_part(lc, s->kw, s->ctl, s->bufs, s->itab, s->epoch, b, s->nnz_bound, 1, pe.slot);
    pe.done();
    if (n < 0) return cuda_ok(cudaGetLastError());
  }
  s->counters.branch_passes++;
  s->counters.kernel_launches += 2;
  const uint64_t nb = s->nnz_bound * 2;
  s->nnz_bound = nb < s->capacity ? nb : s->capacity;
  return SPS_OK;
}

// The passes [pi, end) of a run whose amplitude-only attempt was just enqueued
// (its branching and layer passes, then the phase-only pass it walks, if any),
// as one cooperative launch. Returns false, with nothing enqueued or changed,
// when the run does not fit that launch; the host bookkeeping (serials,
// epochs, label-mask buffers, bounds, counters) is that of the separate
// launches.
static bool launch_fallback_chain(sps_state* s, const LaunchCfg& lc, const ApplyPlan& P,
                                  size_t pi, size_t end, double prune_eps, uint32_t limit,
                                  sps_status* err) {
  *err = SPS_OK;
  const std::vector<Pass>& passes = P.passes;
  const size_t amp_end = P.amp_end[pi];
  if (amp_end - pi > kChainSteps) return false;
  for (size_t k = pi; k < amp_end; ++k)
    if (!(passes[k].kind == PASS_LAYER || (passes[k].kind == PASS_BRANCH && !passes[k].br.pauli)))
      return false;
  const bool has_walk = end > amp_end;
  if (has_walk && !P.amp_walk[pi] && P.amp_par[pi].empty()) return false;
  if (P.amp_par[pi].size() > 2 * kMaxAmpParity) return false;
  ChainStepDesc steps[kChainSteps];
  uint32_t nsteps = 0;
  const uint32_t first_serial = s->pass_serial + 1;
  for (size_t k = pi; k < amp_end; ++k) {
    const Pass& q = passes[k];
    ChainStepDesc& d = steps[nsteps++];
    std::memset(&d, 0, sizeof(d));
    const uint32_t serial = ++s->pass_serial;
    const uint64_t tag = ((uint64_t)s->apply_serial << 32) | (q.first_gate & 0xFFFFFFFFull);
    const sps_status es = next_epoch(s, lc);   // a wrap clears the table before the launch
    if (es != SPS_OK) {
      *err = es;
      return true;
    }
    d.kind = q.kind;
    d.epoch = s->epoch;
    if (q.kind == PASS_LAYER) {
      LayerLaunch& l = d.lay;
      l.fallback = 1;
      l.d = (uint32_t)q.lay.size();
      for (uint32_t j = 0; j < l.d; ++j) l.ops[j] = q.lay[j];
      l.eps = prune_eps;
      l.load_pct = s->load_pct;
      l.max_log2 = s->itab_log2;
      l.pass_serial = serial;
      l.mg = s->masks.writer();
      l.capacity = s->capacity;
      l.fail_tag = tag;
      s->nnz_bound = bound_after(q, s->nnz_bound, s->capacity);
    } else {
      BranchLaunch& b = d.br;
      b.op = q.br;
      b.eps = prune_eps;
      b.load_pct = s->load_pct;
      b.max_log2 = s->itab_log2;
      b.probe_limit = limit;
      b.pass_serial = serial;
      b.coop = s->coop;
      b.capacity = s->capacity;
      b.fail_tag = tag;
      b.mg = s->masks.writer();
      b.fallback = 1;
      const uint64_t nb = s->nnz_bound * 2;
      s->nnz_bound = nb < s->capacity ? nb : s->capacity;
    }
    s->counters.branch_passes++;
  }
  ChainWalk w;
  std::memset(&w, 0, sizeof(w));
  if (has_walk) {
    const Pass& f = passes[amp_end];
    ++s->pass_serial;
    w.ngates = f.ngates;
    if (P.amp_walk[pi]) {
      w.words = reinterpret_cast<const OpWord*>(s->arena + P.run_off[amp_end]);
      w.ftab = reinterpret_cast<const double*>(s->arena + P.ph_off[amp_end]);
      w.nwords = (uint32_t)f.words.size();
      w.has_phase = f.has_phase ? 1u : 0u;
    } else {
      w.par = P.amp_par[pi].data();
      w.npar = (uint32_t)(P.amp_par[pi].size() / 2);
    }
    s->counters.fused_passes++;
  }
  ProfScope ps(s, 11, first_serial, nsteps, 3u);
  const int n = launch_chain(lc, s->kw, s->ctl, s->bufs, s->itab, steps, nsteps, w, s->nnz_bound,
                             ps.slot);
  ps.done();
  // (0, a run too large for the launch, was ruled out above)
  if (n <= 0) *err = SPS_ERR_CUDA;
  s->counters.kernel_launches += 1;
  return true;
}

static uint32_t probe_limit_of(const sps_state* s) {
  return s->probe_limit ? s->probe_limit
                        : (uint32_t)(s->table_slots > 0xFFFFFFFFull ? 0xFFFFFFFFu : s->table_slots);
}

// Options the compiled plan and its image depend on.
static std::vector<uint64_t> plan_options(const sps_state* s) {
  return {s->nqubits, (uint64_t)s->kw, s->capacity, s->max_fused_ops, s->expand ? 1ull : 0ull,
          s->fold ? 1ull : 0ull, s->small_cap, s->bitslice_min_ops, s->bitslice_min_nnz,
          s->commute ? 1ull : 0ull, s->layer_max, s->expand_walk ? 1ull : 0ull,
          s->amp ? 1ull : 0ull};
}

static bool plan_matches(const ApplyPlan& p, const sps_state* s, const sps_gate* gates,
                         size_t ngates, uint64_t eps_bits, const std::vector<uint64_t>& opts) {
  return p.gates.size() == ngates && p.eps_bits == eps_bits && p.bound_in == s->nnz_bound &&
         p.kb_in.known[0] == s->kb.known[0] && p.kb_in.known[1] == s->kb.known[1] &&
         p.kb_in.val[0] == s->kb.val[0] && p.kb_in.val[1] == s->kb.val[1] && p.opts == opts &&
         (ngates == 0 || std::memcmp(p.gates.data(), gates, ngates * sizeof(sps_gate)) == 0);
}

// Compiles an apply: passes, small-state segments, bit-sliced plans and the
// arena image. Small-run records hold each pass's index in the apply (+1) and
// its first gate; the kernel adds the launch's serial base and apply serial.
static sps_status build_plan(sps_state* s, const sps_gate* gates, size_t ngates, double prune_eps,
                             ApplyPlan* P, size_t* bad) {
  P->kb_out = s->kb;
  std::vector<sps_gate> rewritten;
  std::vector<size_t> origin;
  if (s->commute) {
    const sps_status rs = commute_gates(gates, ngates, s->nqubits, &rewritten, &origin, bad);
    if (rs != SPS_OK) return rs;
    gates = rewritten.data();
    ngates = rewritten.size();
  }
  const sps_status cs = compile(gates, ngates, s->nqubits, s->max_fused_ops, &P->passes, bad,
                                &P->kb_out, s->expand, s->fold, s->layer_max);
  if (cs != SPS_OK) return cs;
  // layers that a one-block run would take go back to one pass per gate (the
  // one-block engine runs passes, the layer kernels are whole-GPU)
  if (s->small_cap) {
    std::vector<Pass> split;
    uint64_t b = s->nnz_bound;
    for (Pass& p : P->passes) {
      if (p.kind == PASS_LAYER && b <= s->small_cap) {
        for (size_t j = 0; j < p.lay.size(); ++j) {
          Pass q;
          q.kind = PASS_BRANCH;
          q.first_gate = p.lay_gate[j];
          q.br = p.lay[j];
          b = bound_after(q, b, s->capacity);
          split.push_back(std::move(q));
        }
        continue;
      }
      b = bound_after(p, b, s->capacity);
      split.push_back(std::move(p));
    }
    P->passes.swap(split);
  }
  if (s->commute) {   // failures name the caller's gate
    for (Pass& p : P->passes) {
      p.first_gate = origin[p.first_gate];
      for (uint64_t& g : p.lay_gate) g = origin[g];
    }
  }
  const std::vector<Pass>& passes = P->passes;
  const size_t np = passes.size();
  // 1. segments of consecutive passes that a small-state run can take: the
  //    nonzero bound (doubling per branching pass) stays within small_cap
  P->seg_end.assign(np, 0);
  P->bound_at.assign(np, 0);
  {
    uint64_t b = s->nnz_bound;
    for (size_t i = 0; i < np; ++i) {
      P->bound_at[i] = b;
      b = bound_after(passes[i], b, s->capacity);
    }
    b = s->nnz_bound;
    for (size_t i = 0; i < np;) {
      if (s->small_cap && b <= s->small_cap) {
        size_t j = i;
        uint64_t bb = b;
        while (j < np && passes[j].kind != PASS_EXPAND) {
          const uint64_t after = bound_after(passes[j], bb, s->capacity);
          if (after > s->small_cap) break;
          bb = after;
          ++j;
        }
        if (j > i) {
          P->seg_end[i] = j;
          b = bb;
          i = j;
          continue;
        }
      }
      b = bound_after(passes[i], b, s->capacity);
      ++i;
    }
  }
  // 2a. runs of branching passes on pairwise disjoint qubits (targets and
  //     controls), up to kMaxAmpGates gates, outside small runs: one
  //     amplitude-only attempt each
  P->amp_end.assign(np, 0);
  if (s->amp) {
    auto branching = [&](const Pass& q) {
      return (q.kind == PASS_BRANCH && !q.br.pauli) || q.kind == PASS_LAYER;
    };
    for (size_t i = 0; i < np;) {
      if (P->seg_end[i]) {
        i = P->seg_end[i];
        continue;
      }
      if (!branching(passes[i])) {
        ++i;
        continue;
      }
      uint64_t sup0 = 0, sup1 = 0;
      uint32_t gates = 0;
      size_t j = i;
      while (j < np && !P->seg_end[j] && branching(passes[j])) {
        const Pass& q = passes[j];
        uint64_t q0 = 0, q1 = 0;
        uint32_t g = 0;
        auto add = [&](const BranchOp& op) {
          q0 |= op.c[0] | op.m[0];
          q1 |= op.c[1] | op.m[1];
          ++g;
        };
        if (q.kind == PASS_BRANCH) add(q.br);
        else for (const BranchOp& op : q.lay) add(op);
        if (gates + g > kMaxAmpGates || (q0 & sup0) || (q1 & sup1)) break;
        sup0 |= q0;
        sup1 |= q1;
        gates += g;
        ++j;
      }
      P->amp_end[i] = j;
      i = j;
    }
  }
  // A run long enough, on a state large enough, for the bit-sliced form is
  // faster as that separate pass than walked on each output, unless it holds
  // only signs (Z and controlled Z: pi steps, no selector, no flip, no
  // arbitrary phase): then the attempt applies it as a parity of conditions.
  P->amp_walk.assign(np, 0);
  P->amp_par.assign(np, std::vector<uint64_t>());
  std::vector<uint8_t> amp_walked(np, 0);   // fused passes walked by an attempt
  for (size_t i = 0; i < np; ++i) {
    const size_t j = P->amp_end[i];
    if (!j || j >= np) continue;
    const Pass& f = passes[j];
    if (f.kind != PASS_FUSED || f.has_perm || P->seg_end[j]) continue;
    const bool sliced = s->bitslice_min_ops && f.ops.size() >= s->bitslice_min_ops &&
                        P->bound_at[j] >= s->bitslice_min_nnz;
    if (!sliced) {
      P->amp_walk[i] = 1;
      amp_walked[j] = 1;
      continue;
    }
    std::vector<uint64_t> par;
    bool signs = true;
    for (const FOp& o : f.ops) {
      if ((o.t[0] | o.t[1]) || o.ph != NO_PH || (o.a0 & 3u) || (o.a1 & 3u)) {
        signs = false;
        break;
      }
      // sign steps s0, s1 (pi or none) for sel = 0 / 1: the sign flips where
      // c and (s0 xor (sel and (s0 xor s1))) hold, i.e. the parity of "c" (if
      // s0) and "c and the selector bit" (if s0 != s1)
      const bool s0 = (o.a0 & 7u) == 4u;
      const bool s1 = o.sbit != NO_SEL && (o.a1 & 7u) == 4u;
      if (s0) {
        par.push_back(o.c[0]);
        par.push_back(o.c[1]);
      }
      if (o.sbit != NO_SEL && s0 != s1) {
        uint64_t sb[2] = {0ull, 0ull};
        sb[o.sbit >> 6] = 1ull << (o.sbit & 63u);
        par.push_back(o.c[0] | sb[0]);
        par.push_back(o.c[1] | sb[1]);
      }
    }
    if (signs && par.size() <= 2 * kMaxAmpParity && f.ngates > 0) P->amp_par[i] = std::move(par);
  }
  // 2b. an expansion takes the fused run right after it (outside small runs),
  //    unless that run is long enough and the state large enough for the
  //    bit-sliced form (faster there than the per-label walk)
  P->walk_next.assign(np, 0);
  if (s->expand_walk)
    for (size_t i = 0; i + 1 < np; ++i) {
      const Pass& f = passes[i + 1];
      const bool sliced = s->bitslice_min_ops && f.ops.size() >= s->bitslice_min_ops &&
                          P->bound_at[i + 1] >= s->bitslice_min_nnz;
      if (passes[i].kind == PASS_EXPAND && !P->seg_end[i] && f.kind == PASS_FUSED &&
          !P->seg_end[i + 1] && !sliced)
        P->walk_next[i] = 1;
    }
  // 3. device data: bit-sliced plans of long fused runs outside small runs,
  //    then the op streams, tables and small-run records
  P->bs.assign(np, BsPass());
  P->bs_off.assign(np, 0);
  P->bs_tab.assign(np, 0);
  P->bs_tab_entries = 0;
  P->run_off.assign(np, 0);
  P->ph_off.assign(np, 0);
  size_t bs_bytes = 0;
  for (size_t i = 0; i < np;) {
    if (P->seg_end[i]) {
      i = P->seg_end[i];
      continue;
    }
    const Pass& p = passes[i];
    // a run walked by an expansion or by an amplitude-only attempt stays in the
    // direct form (the walk is the direct form's arithmetic)
    const bool walked = (i > 0 && P->walk_next[i - 1]) || amp_walked[i];
    if (p.kind == PASS_FUSED && !walked && s->bitslice_min_ops && p.ops.size() >= s->bitslice_min_ops &&
        P->bound_at[i] >= s->bitslice_min_nnz) {
      build_bitslice(p, s->nqubits, &P->bs[i]);
      if (P->bs[i].op_words() > kBsMaxOps) {   // too long for one launch: direct form
        P->bs[i] = BsPass();
      } else {
        P->bs_off[i] = bs_bytes;
        bs_bytes += align16(P->bs[i].factors.size() * 8);
        P->bs_tab[i] = P->bs_tab_entries;
        P->bs_tab_entries += P->bs[i].table_entries();
      }
    }
    ++i;
  }
  // an expansion from |0...0> and the bit-sliced run after it, as one launch
  // (taken at apply time when the reset is still pending)
  P->bs_ex_ok = false;
  if (np >= 2 && s->bs_jit != 0 && passes[0].kind == PASS_EXPAND && !P->seg_end[0] &&
      passes[1].kind == PASS_FUSED && !P->seg_end[1] && !P->bs[1].ops.empty() &&
      s->nnz_bound == 1 && passes[0].ex_d < 63 && (1ull << passes[0].ex_d) <= s->capacity &&
      (s->bs_jit == 2 || (1ull << passes[0].ex_d) >= kBsJitMinNnz) &&
      build_bitslice_expand(passes[0], passes[1], s->nqubits, prune_eps, &P->bs_ex)) {
    P->bs_ex_ok = true;
    P->bs_ex_off = bs_bytes;
    bs_bytes += align16(P->bs_ex.factors.size() * 8);
    P->bs_ex_tab = P->bs_tab_entries;
    P->bs_tab_entries += P->bs_ex.table_entries();
  }
  std::vector<unsigned char>& img = P->image;
  img.assign(bs_bytes, 0);
  for (size_t i = 0; i < np; ++i) {
    const BsPass& b = P->bs[i];
    if (b.ops.empty() || b.factors.empty()) continue;
    std::memcpy(img.data() + P->bs_off[i], b.factors.data(), b.factors.size() * 8);
  }
  if (P->bs_ex_ok && !P->bs_ex.factors.empty())
    std::memcpy(img.data() + P->bs_ex_off, P->bs_ex.factors.data(), P->bs_ex.factors.size() * 8);
  auto put = [&](const void* src, size_t bytes) {
    const size_t at = img.size();
    img.resize(align16(at + bytes), 0);
    std::memcpy(img.data() + at, src, bytes);
    return at;
  };
  for (size_t i = 0; i < np;) {
    if (!P->seg_end[i]) {
      const Pass& p = passes[i];
      if (p.kind == PASS_FUSED && P->bs[i].ops.empty()) {   // direct fused pass
        P->run_off[i] = put(p.words.data(), p.words.size() * sizeof(OpWord));
        if (!p.ftab.empty()) P->ph_off[i] = put(p.ftab.data(), p.ftab.size() * sizeof(double));
      }
      if (p.kind == PASS_EXPAND) {   // factor tables, then mask tables
        P->run_off[i] = put(p.ex_f.data(), p.ex_f.size() * sizeof(double));
        P->ph_off[i] = put(p.ex_m.data(), p.ex_m.size() * sizeof(uint64_t));
      }
      ++i;
      continue;
    }
    const size_t j = P->seg_end[i];
    std::vector<RunPass> recs(j - i);
    for (size_t k = i; k < j; ++k) {
      const Pass& p = passes[k];
      RunPass& r = recs[k - i];
      std::memset(&r, 0, sizeof(r));
      r.kind = p.kind;
      r.pass_serial = (uint32_t)(k + 1);
      r.fail_tag = p.first_gate & 0xFFFFFFFFull;
      r.eps2 = prune_eps * prune_eps;
      r.eps = prune_eps;
      if (p.kind == PASS_FUSED) {
        r.nops = p.ngates;
        r.nwords = (uint32_t)p.words.size();
        r.flags = (p.has_perm ? 1u : 0u) | (p.has_phase ? 2u : 0u);
        r.ops_off = (uint32_t)put(p.words.data(), p.words.size() * sizeof(OpWord));
        r.ph_off = p.ftab.empty() ? 0u : (uint32_t)put(p.ftab.data(), p.ftab.size() * sizeof(double));
      } else {
        r.br_off = (uint32_t)put(&p.br, sizeof(BranchOp));
      }
    }
    P->run_off[i] = put(recs.data(), recs.size() * sizeof(RunPass));
    i = j;
  }
  return SPS_OK;
}

sps_status sps_apply(sps_state* s, const sps_gate* gates, size_t ngates, double prune_eps,
                     size_t* failed_gate) {
  if (!s || (ngates && !gates) || !(prune_eps >= 0.0)) return SPS_ERR_ARG;
  ++s->version;
  uint64_t eps_bits;
  std::memcpy(&eps_bits, &prune_eps, sizeof(eps_bits));
  std::vector<uint64_t> opts = plan_options(s);
  if (!s->plan_cache || !s->plan || !plan_matches(*s->plan, s, gates, ngates, eps_bits, opts)) {
    std::unique_ptr<ApplyPlan> np(new (std::nothrow) ApplyPlan());
    if (!np) return SPS_ERR_OOM;
    size_t bad = 0;
    const sps_status cs = build_plan(s, gates, ngates, prune_eps, np.get(), &bad);
    if (cs != SPS_OK) {
      if (failed_gate) *failed_gate = bad;
      return cs;
    }
    np->gates.assign(gates, gates + ngates);
    np->eps_bits = eps_bits;
    np->kb_in = s->kb;
    np->bound_in = s->nnz_bound;
    np->opts = std::move(opts);
    s->plan = std::move(np);
    s->plan_resident = false;
  }
  const ApplyPlan& P = *s->plan;
  const bool build_tables = !s->plan_resident;   // a plan new to the device
  if (build_tables && P.bs_tab_entries) {
    const sps_status ts = ensure_bs_tables(s, (size_t)P.bs_tab_entries * 16);
    if (ts != SPS_OK) return ts;
  }
  if (!s->plan_resident && !P.image.empty()) {
    const sps_status as = ensure_arena(s, P.image.size());
    if (as != SPS_OK) return as;
    sps_state::Staging* stg = nullptr;
    const sps_status ss = take_staging(s, P.image.size(), &stg);
    if (ss != SPS_OK) return ss;
    std::memcpy(stg->host, P.image.data(), P.image.size());
    // runs in stream order after earlier kernels that read the arena
    if (cudaMemcpyAsync(s->arena, stg->host, P.image.size(), cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess ||
        cudaEventRecord(stg->copied, s->stream) != cudaSuccess)
      return cuda_ok(cudaGetLastError());
    stg->pending = true;
    s->counters.upload_bytes += P.image.size();
  }
  s->plan_resident = true;
  s->kb = P.kb_out;
  const std::vector<Pass>& passes = P.passes;
  const std::vector<size_t>& seg_end = P.seg_end;
  const std::vector<BsPass>& bs = P.bs;
  const std::vector<size_t>& bs_off = P.bs_off;
  const std::vector<size_t>& run_off = P.run_off;
  const std::vector<size_t>& ph_off = P.ph_off;
  const LaunchCfg lc = cfg_of(s);
  const uint32_t limit = s->probe_limit ? s->probe_limit : (uint32_t)(s->table_slots > 0xFFFFFFFFull ? 0xFFFFFFFFu : s->table_slots);
  const uint32_t serial_base = s->pass_serial;
  ++s->apply_serial;
  size_t amp_run_end = 0;   // passes before this index belong to an attempted run
  // a pending reset is taken by a leading expansion pass, else enqueued now
  bool from_reset = false;
  if (s->reset_pending) {
    if (!passes.empty() && passes[0].kind == PASS_EXPAND && !seg_end[0]) {
      from_reset = true;
      s->reset_pending = false;
    } else {
      const sps_status fs = flush_reset(s);
      if (fs != SPS_OK) return fs;
    }
  }
  for (size_t pi = 0; pi < passes.size(); ++pi) {
    const Pass& p = passes[pi];
    if (seg_end[pi]) {
      const size_t j = seg_end[pi];
      uint32_t nbranch = 0;
      for (size_t k = pi; k < j; ++k) nbranch += passes[k].kind == PASS_BRANCH ? 1u : 0u;
      ProfScope ps(s, 4, s->pass_serial + 1, (uint32_t)(j - pi), 3u);
      const int n = launch_small_run(s->stream, s->kw, s->ctl, s->bufs, s->arena,
                                     (uint32_t)run_off[pi], (uint32_t)(j - pi), s->capacity,
                                     s->masks.writer(), serial_base, s->apply_serial, ps.slot);
      ps.done();
      if (n < 0) return cuda_ok(cudaGetLastError());
      s->amp_force = true;   // the run moves labels
      s->pass_serial += (uint32_t)(j - pi);
      s->counters.branch_passes += nbranch;
      s->counters.fused_passes += (j - pi) - nbranch;
      s->counters.kernel_launches += 1;
      for (uint32_t k = 0; k < nbranch; ++k) {
        const uint64_t nb = s->nnz_bound * 2;
        s->nnz_bound = nb < s->capacity ? nb : s->capacity;
      }
      pi = j - 1;
      continue;
    }
    const bool scatter = s->branch_form == 1 || s->capacity >= (1ull << 32);
    if (P.amp_end[pi] && !scatter) {   // a run's attempt, then its passes as fallbacks
      BranchOp ops[kMaxAmpGates];
      uint32_t d = 0;
      for (size_t k = pi; k < P.amp_end[pi]; ++k) {
        if (passes[k].kind == PASS_BRANCH) ops[d++] = passes[k].br;
        else for (const BranchOp& op : passes[k].lay) ops[d++] = op;
      }
      const uint64_t tg = ((uint64_t)s->apply_serial << 32) | (p.first_gate & 0xFFFFFFFFull);
      const Pass* walk = nullptr;
      const OpWord* words = nullptr;
      const double* ftab = nullptr;
      const std::vector<uint64_t>* par = nullptr;
      if (P.amp_walk[pi]) {
        const size_t j = P.amp_end[pi];
        walk = &passes[j];
        words = reinterpret_cast<const OpWord*>(s->arena + run_off[j]);
        ftab = reinterpret_cast<const double*>(s->arena + ph_off[j]);
      } else if (!P.amp_par[pi].empty()) {
        walk = &passes[P.amp_end[pi]];
        par = &P.amp_par[pi];
      }
      const sps_status as = launch_amp_attempt(s, lc, ops, d, prune_eps, s->pass_serial + 1, tg,
                                               walk, words, ftab, par);
      if (as != SPS_OK) return as;
      amp_run_end = P.amp_end[pi] + (walk ? 1 : 0);
      sps_status cs = SPS_OK;
      if (s->chain && launch_fallback_chain(s, lc, P, pi, amp_run_end, prune_eps, limit, &cs)) {
        if (cs != SPS_OK) return cs;
        pi = amp_run_end - 1;
        continue;
      }
    }
    const uint32_t fb = pi < amp_run_end ? 1u : 0u;   // a fallback pass of an attempted run
    if (!fb && (p.kind == PASS_BRANCH || p.kind == PASS_LAYER)) s->amp_force = true;
    const uint32_t serial = ++s->pass_serial;
    const uint64_t tag = ((uint64_t)s->apply_serial << 32) | (p.first_gate & 0xFFFFFFFFull);
    if (p.kind == PASS_EXPAND && pi == 0 && from_reset && P.bs_ex_ok) {
      // the expansion and the bit-sliced run after it in one compiled launch
      const Pass& f = passes[1];
      BsLaunch bl;
      bl.plan = &P.bs_ex;
      bl.factors = reinterpret_cast<const long long*>(s->arena + P.bs_ex_off);
      bl.tables = s->bs_tables + 2 * P.bs_ex_tab;
      bl.build_tables = build_tables ? 1u : 0u;
      bl.ngates = f.ngates;
      bl.has_perm = 1u;
      bl.has_phase = P.bs_ex.aux_bits > 0 ? 1u : 0u;
      bl.groups = 0;
      MaskRing ring = s->masks;   // taken only if the launch happens
      bl.mg = ring.writer();
      bl.fallback = 0;
      ReadoutFuse rf;
      uint32_t rd_done = 0;
      if (s->rd_on && passes.size() == 2) {   // the launch ends the apply
        std::memcpy(rf.mask, s->rd_mask, sizeof(rf.mask));
        std::memcpy(rf.value, s->rd_value, sizeof(rf.value));
        rf.part = s->rd_buf;
        rf.out = s->rd_buf + s->rd_cap;
        rf.cap = s->rd_cap;
        rf.min_planes = s->rd_min_planes;
        bl.rd = &rf;
        bl.rd_done = &rd_done;
      }
      const uint64_t nout = 1ull << p.ex_d;
      ProfScope ps(s, 7, serial, p.ex_d, 3u | 4u | 8u | 16u);
      const int n = launch_fused_bs_jit(lc, s->kw, s->ctl, s->bufs, bl, nout, ps.slot);
      if (rd_done) ps.rec.flags |= 32u;
      ps.done();
      if (n < 0) return cuda_ok(cudaGetLastError());
      if (n > 0 && rd_done) s->rd_version = s->version;
      if (n > 0) {
        s->masks = ring;
        s->amp_force = true;
        s->counters.branch_passes++;
        s->counters.fused_passes++;
        s->counters.kernel_launches += (uint64_t)n;
        s->nnz_bound = nout;
        ++s->pass_serial;   // the run's pass serial
        ++pi;
        continue;
      }
      // the compiled form is not available: the two passes as usual
    }
    if (p.kind == PASS_EXPAND) {
      ExpandLaunch e;
      e.f = reinterpret_cast<const double*>(s->arena + run_off[pi]);
      e.m = reinterpret_cast<const uint64_t*>(s->arena + ph_off[pi]);
      e.d = p.ex_d;
      e.real = p.ex_real ? 1u : 0u;
      e.pass_serial = serial;
      e.mg = s->masks.writer();
      e.eps = prune_eps;
      e.capacity = s->capacity;
      e.fail_tag = tag;
      e.words = nullptr;
      e.ftab = nullptr;
      e.nwords = 0;
      e.fused_gates = 0;
      e.has_phase = 0;
      e.from_reset = from_reset && pi == 0 ? 1u : 0u;
      const bool walk = P.walk_next[pi] != 0;
      if (walk) {   // the fused run after the expansion, applied before the stores
        const Pass& f = passes[pi + 1];
        e.words = reinterpret_cast<const OpWord*>(s->arena + run_off[pi + 1]);
        e.ftab = reinterpret_cast<const double*>(s->arena + ph_off[pi + 1]);
        e.nwords = (uint32_t)f.words.size();
        e.fused_gates = f.ngates;
        e.has_phase = f.has_phase ? 1u : 0u;
      }
      ProfScope ps(s, 7, serial, p.ex_d, P.walk_next[pi] ? 7u : 3u);
      const int n = launch_expand(lc, s->kw, s->ctl, s->bufs, e, s->nnz_bound, ps.slot);
      ps.done();
      if (n < 0) return cuda_ok(cudaGetLastError());
      s->amp_force = true;
      s->counters.branch_passes++;
      s->counters.kernel_launches += 1;
      s->nnz_bound = bound_after(p, s->nnz_bound, s->capacity);
      if (walk) {   // the fused pass is done: keep the pass serials in step
        ++s->pass_serial;
        s->counters.fused_passes++;
        ++pi;
      }
      continue;
    }
    if (p.kind == PASS_LAYER) {
      if (scatter) {   // the layer kernels are gather-form: one pass per gate
        for (size_t j = 0; j < p.lay.size(); ++j) {
          const uint64_t tg = ((uint64_t)s->apply_serial << 32) | (p.lay_gate[j] & 0xFFFFFFFFull);
          const sps_status bs2 = launch_branch_pass(s, lc, p.lay[j], prune_eps,
                                                    j ? ++s->pass_serial : serial, tg, limit);
          if (bs2 != SPS_OK) return bs2;
        }
        continue;
      }
      const sps_status es = next_epoch(s, lc);
      if (es != SPS_OK) return es;
      LayerLaunch l;
      std::memset(&l, 0, sizeof(l));
      l.fallback = fb;
      l.d = (uint32_t)p.lay.size();
      for (uint32_t j = 0; j < l.d; ++j) l.ops[j] = p.lay[j];
      l.eps = prune_eps;
      l.load_pct = s->load_pct;
      l.max_log2 = s->itab_log2;
      l.pass_serial = serial;
      l.mg = s->masks.writer();
      l.capacity = s->capacity;
      l.fail_tag = tag;
      ProfScope pb(s, 5, serial, l.d, 3u);
      int n = launch_layer_part(lc, s->kw, s->ctl, s->bufs, s->itab, s->epoch, l, s->nnz_bound, 0, pb.slot);
      pb.done();
      if (n < 0) return cuda_ok(cudaGetLastError());
      ProfScope pe(s, 6, serial, l.d, 3u);
      n = launch_layer_part(lc, s->kw, s->ctl, s->bufs, s->itab, s->epoch, l, s->nnz_bound, 1, pe.slot);
      pe.done();
      if (n < 0) return cuda_ok(cudaGetLastError());
      s->counters.branch_passes++;
      s->counters.kernel_launches += 2;
      s->nnz_bound = bound_after(p, s->nnz_bound, s->capacity);
      continue;
    }
    if (p.kind == PASS_FUSED) {
      const uint32_t flags = (p.has_perm ? 1u : 0u) | (p.has_phase ? 2u : 0u);
      ProfScope ps(s, 1, serial, (uint32_t)p.ops.size(), flags);
      int n;
      if (!bs[pi].ops.empty()) {
        BsLaunch bl;
        bl.plan = &bs[pi];
        bl.factors = reinterpret_cast<const long long*>(s->arena + bs_off[pi]);
        bl.tables = s->bs_tables + 2 * P.bs_tab[pi];
        bl.build_tables = build_tables ? 1u : 0u;
        bl.ngates = p.ngates;
        bl.has_perm = p.has_perm;
        bl.has_phase = p.has_phase;
        bl.groups = s->bs_groups;
        bl.mg = p.has_perm ? s->masks.writer() : 0u;
        bl.fallback = fb;
        n = 0;
        if (s->bs_jit == 2 || (s->bs_jit == 1 && s->nnz_bound >= kBsJitMinNnz)) {
          n = launch_fused_bs_jit(lc, s->kw, s->ctl, s->bufs, bl, s->nnz_bound, ps.slot);
          if (n > 0) ps.rec.flags |= 16u;   // the form compiled for this run
        }
        if (n == 0) n = launch_fused_bs(lc, s->kw, s->ctl, s->bufs, bl, s->nnz_bound, ps.slot);
        if (n == 0) n = -1;   // the plan was checked to fit one launch
        ps.rec.flags |= 8u;   // bit-sliced
      } else {
        n = launch_fused(lc, s->kw, s->ctl, s->bufs, p,
                         reinterpret_cast<const OpWord*>(s->arena + run_off[pi]),
                         reinterpret_cast<const double*>(s->arena + ph_off[pi]), s->nnz_bound,
                         p.has_perm ? s->masks.writer() : 0u, s->fused_labels, fb, ps.slot);
      }
      ps.done();
      if (n < 0) return cuda_ok(cudaGetLastError());
      if (p.has_perm) s->amp_force = true;   // labels changed in place
      s->counters.fused_passes++;
      s->counters.kernel_launches += (uint64_t)n;
    } else {
      const sps_status bs2 = launch_branch_pass(s, lc, p.br, prune_eps, serial, tag, limit, fb);
      if (bs2 != SPS_OK) return bs2;
    }
  }
  s->counters.gates += ngates;
  return SPS_OK;
}

sps_status sps_sync(sps_state* s, size_t* failed_gate) {
  if (!s) return SPS_ERR_ARG;
  sps_status st = read_ctl(s);
  if (st != SPS_OK) return st;
  const Ctl c = *s->ctl_host;
  s->nnz_bound = c.nnz > 0 ? c.nnz : 1;
  if (c.status == 0u) return SPS_OK;
  if (failed_gate) *failed_gate = (size_t)(c.fail_gate & 0xFFFFFFFFull);
  // recover: clear the error and the table; the state is the last good one,
  // which passes enqueued after the failed one no longer describe
  know_nothing(s);
  const LaunchCfg lc = cfg_of(s);
  if (launch_reset_status(s->stream, s->ctl) < 0 ||
      (s->table && launch_table_clear(lc, s->table, s->table_slots) < 0))
    return cuda_ok(cudaGetLastError());
  s->counters.kernel_launches += 2;
  st = cuda_ok(cudaStreamSynchronize(s->stream));
  if (st != SPS_OK) return st;
  return (sps_status)c.status;
}

sps_status sps_get_updates(sps_state* s, uint64_t* updates) {
  if (!s || !updates) return SPS_ERR_ARG;
  const sps_status st = sps_sync(s, nullptr);
  if (st != SPS_OK) return st;
  *updates = s->ctl_host->updates;
  return SPS_OK;
}

sps_status sps_nnz(sps_state* s, uint64_t* nnz) {
  if (!s || !nnz) return SPS_ERR_ARG;
  const sps_status st = sps_sync(s, nullptr);
  if (st != SPS_OK) return st;
  *nnz = s->ctl_host->nnz;
  return SPS_OK;
}

sps_status sps_get_amplitudes(sps_state* s, uint64_t* key_hi, uint64_t* key_lo, double* re,
                              double* im, uint64_t cap, uint64_t* nnz_out) {
  if (!s || !key_lo || !re || !im || !nnz_out) return SPS_ERR_ARG;
  sps_status st = sps_sync(s, nullptr);
  if (st != SPS_OK) return st;
  const uint64_t n = s->ctl_host->nnz;
  *nnz_out = n;
  if (n > cap) return SPS_ERR_CAPACITY;
  if (n == 0) return SPS_OK;
  const SoA b = s->bufs.b[s->ctl_host->cur];
  bool ok = cudaMemcpyAsync(key_lo, b.lo, n * 8, cudaMemcpyDefault, s->stream) == cudaSuccess &&
            cudaMemcpyAsync(re, b.re, n * 8, cudaMemcpyDefault, s->stream) == cudaSuccess &&
            cudaMemcpyAsync(im, b.im, n * 8, cudaMemcpyDefault, s->stream) == cudaSuccess;
  if (ok && key_hi) {
    if (s->kw == 2) {
      ok = cudaMemcpyAsync(key_hi, b.hi, n * 8, cudaMemcpyDefault, s->stream) == cudaSuccess;
    } else if (is_device_pointer(key_hi)) {
      ok = cudaMemsetAsync(key_hi, 0, n * 8, s->stream) == cudaSuccess;
    } else {
      std::memset(key_hi, 0, n * 8);
    }
  }
  if (!ok) return cuda_ok(cudaGetLastError());
  return cuda_ok(cudaStreamSynchronize(s->stream));
}

sps_status sps_set_amplitudes(sps_state* s, const uint64_t* key_hi, const uint64_t* key_lo,
                              const double* re, const double* im, uint64_t n) {
  if (!s || (n && (!key_lo || !re || !im))) return SPS_ERR_ARG;
  if (n > s->capacity) return SPS_ERR_CAPACITY;
  ++s->version;
  s->amp_force = true;
  sps_status st = sps_sync(s, nullptr);
  if (st != SPS_OK) return st;
  const SoA b = s->bufs.b[0];
  bool ok = true;
  if (n) {
    ok = cudaMemcpyAsync(b.lo, key_lo, n * 8, cudaMemcpyDefault, s->stream) == cudaSuccess &&
         cudaMemcpyAsync(b.re, re, n * 8, cudaMemcpyDefault, s->stream) == cudaSuccess &&
         cudaMemcpyAsync(b.im, im, n * 8, cudaMemcpyDefault, s->stream) == cudaSuccess;
    if (ok && s->kw == 2) {
      ok = key_hi ? cudaMemcpyAsync(b.hi, key_hi, n * 8, cudaMemcpyDefault, s->stream) == cudaSuccess
                  : cudaMemsetAsync(b.hi, 0, n * 8, s->stream) == cudaSuccess;
    }
  }
  if (!ok) return cuda_ok(cudaGetLastError());
  uint64_t lim0, lim1;
  label_limits(s->nqubits, &lim0, &lim1);
  // For 64-bit labels the high words must be zero: check them from the spare buffer.
  Bufs chk = s->bufs;
  if (s->kw == 1 && key_hi && n) {
    if (cudaMemcpyAsync(s->bufs.b[1].lo, key_hi, n * 8, cudaMemcpyDefault, s->stream) != cudaSuccess)
      return cuda_ok(cudaGetLastError());
  }
  if (launch_set_nnz(s->stream, s->ctl, n, s->masks.writer()) < 0 ||
      cudaMemsetAsync(s->dflag, 0, sizeof(unsigned), s->stream) != cudaSuccess ||
      launch_check_labels(s->stream, s->kw, s->ctl, chk, lim0, lim1, s->dflag, n,
                          s->masks.writer()) < 0)
    return cuda_ok(cudaGetLastError());
  int launched = 2;
  if (s->kw == 1 && key_hi && n) {
    // labels in bufs[1].lo are the high words; every one must be zero
    Bufs hib = s->bufs;
    hib.b[0].lo = s->bufs.b[1].lo;
    if (launch_check_labels(s->stream, 1, s->ctl, hib, 0ull, 0ull, s->dflag, n, kNoMasks) < 0)
      return cuda_ok(cudaGetLastError());
    ++launched;
  }
  s->counters.kernel_launches += launched;
  if (cudaMemcpyAsync(s->hflag, s->dflag, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream) !=
      cudaSuccess)
    return cuda_ok(cudaGetLastError());
  st = cuda_ok(cudaStreamSynchronize(s->stream));
  if (st != SPS_OK) return st;
  s->nnz_bound = n ? n : 1;
  if (*s->hflag) {
    // reject: fall back to |0...0>
    static const double kOne = 1.0;
    ok = cudaMemsetAsync(b.lo, 0, 8, s->stream) == cudaSuccess &&
         (s->kw == 1 || cudaMemsetAsync(b.hi, 0, 8, s->stream) == cudaSuccess) &&
         cudaMemcpyAsync(b.re, &kOne, 8, cudaMemcpyHostToDevice, s->stream) == cudaSuccess &&
         cudaMemsetAsync(b.im, 0, 8, s->stream) == cudaSuccess && launch_set_nnz(s->stream, s->ctl, 1, s->masks.writer()) >= 0 &&
         cudaStreamSynchronize(s->stream) == cudaSuccess;
    s->nnz_bound = 1;
    s->counters.kernel_launches += 1;
    know_all_zero(s);
    return ok ? SPS_ERR_ARG : cuda_ok(cudaGetLastError());
  }
  return know_from_device(s);
}

// Blocks of a probability readout: about 1,024 entries each (the last block
// adds the block sums in block order, so fewer blocks mean a shorter tail),
// at most prob_blocks.
static int prob_grid(const sps_state* s) {
  const uint64_t b = (s->nnz_bound + 8191) / 8192;
  return b < 1 ? 1 : b > (uint64_t)s->prob_blocks ? s->prob_blocks : (int)b;
}

// The registered readout's sum holds for the state now and this condition.
static bool readout_fused(const sps_state* s, const uint64_t mask[2], const uint64_t value[2]) {
  return s->rd_on && s->rd_version == s->version && !s->reset_pending &&
         s->rd_mask[0] == mask[0] && s->rd_mask[1] == mask[1] && s->rd_value[0] == value[0] &&
         s->rd_value[1] == value[1];
}

sps_status sps_set_readout(sps_state* s, const uint64_t mask[2], const uint64_t value[2]) {
  if (!s || (!mask) != (!value)) return SPS_ERR_ARG;
  if (!mask) {
    s->rd_on = false;
    return SPS_OK;
  }
  if (!s->rd_buf) {
    // one sum per block of the compiled launch: at most 16 resident per SM
    void* p = nullptr;
    const uint32_t cap = (uint32_t)(s->sms > 0 ? s->sms : 1) * 16u;
    const sps_status st = dev_alloc(s, sizeof(double) * (cap + 1), &p);
    if (st != SPS_OK) return st;
    s->rd_buf = (double*)p;
    s->rd_cap = cap;
  }
  const bool same = s->rd_on && s->rd_mask[0] == mask[0] && s->rd_mask[1] == mask[1] &&
                    s->rd_value[0] == value[0] && s->rd_value[1] == value[1];
  if (!same) s->rd_version = 0;   // the sum in rd_buf is for another condition
  std::memcpy(s->rd_mask, mask, sizeof(s->rd_mask));
  std::memcpy(s->rd_value, value, sizeof(s->rd_value));
  s->rd_on = true;
  return SPS_OK;
}

sps_status sps_probability(sps_state* s, const uint64_t mask[2], const uint64_t value[2], double* p) {
  if (!s || !mask || !value || !p) return SPS_ERR_ARG;
  sps_status st = sps_sync(s, nullptr);
  if (st != SPS_OK) return st;
  if (readout_fused(s, mask, value)) {
    s->counters.fused_readouts += 1;
    if (cudaMemcpyAsync(s->hresult, s->rd_buf + s->rd_cap, sizeof(double), cudaMemcpyDeviceToHost,
                        s->stream) != cudaSuccess)
      return cuda_ok(cudaGetLastError());
    st = cuda_ok(cudaStreamSynchronize(s->stream));
    if (st != SPS_OK) return st;
    *p = *s->hresult;
    return SPS_OK;
  }
  const LaunchCfg lc = cfg_of(s);
  ProfScope ps(s, 12, s->pass_serial, 0, 0u);
  const int pn = launch_probability(lc, s->kw, s->ctl, s->bufs, mask[0], mask[1], value[0],
                                    value[1], s->partials, prob_grid(s), s->dresult, ps.slot);
  ps.done();
  if (pn < 0) return cuda_ok(cudaGetLastError());
  s->counters.kernel_launches += 1;
  if (cudaMemcpyAsync(s->hresult, s->dresult, sizeof(double), cudaMemcpyDeviceToHost, s->stream) !=
      cudaSuccess)
    return cuda_ok(cudaGetLastError());
  st = cuda_ok(cudaStreamSynchronize(s->stream));
  if (st != SPS_OK) return st;
  *p = *s->hresult;
  return SPS_OK;
}

sps_status sps_probability_async(sps_state* s, const uint64_t mask[2], const uint64_t value[2],
                                 double* out) {
  if (!s || !mask || !value || !out) return SPS_ERR_ARG;
  if (readout_fused(s, mask, value)) {
    s->counters.fused_readouts += 1;
    if (cudaMemcpyAsync(out, s->rd_buf + s->rd_cap, sizeof(double), cudaMemcpyDefault, s->stream) !=
        cudaSuccess)
      return cuda_ok(cudaGetLastError());
    return SPS_OK;
  }
  const sps_status fs = flush_reset(s);
  if (fs != SPS_OK) return fs;
  const LaunchCfg lc = cfg_of(s);
  ProfScope ps(s, 12, s->pass_serial, 0, 0u);
  const int pn = launch_probability(lc, s->kw, s->ctl, s->bufs, mask[0], mask[1], value[0],
                                    value[1], s->partials, prob_grid(s), s->dresult, ps.slot);
  ps.done();
  if (pn < 0) return cuda_ok(cudaGetLastError());
  s->counters.kernel_launches += 1;
  if (cudaMemcpyAsync(out, s->dresult, sizeof(double), cudaMemcpyDefault, s->stream) != cudaSuccess)
    return cuda_ok(cudaGetLastError());
  return SPS_OK;
}

sps_status sps_pauli_exp(sps_state* s, const uint64_t x[2], const uint64_t z[2],
                         const uint64_t cmask[2], double theta, double prune_eps) {
  if (!s || !x || !z || !cmask || !(prune_eps >= 0.0) || !std::isfinite(theta)) return SPS_ERR_ARG;
  ++s->version;
  uint64_t lim[2];
  label_limits(s->nqubits, &lim[0], &lim[1]);
  for (int w = 0; w < 2; ++w)
    if (((x[w] | z[w] | cmask[w]) & ~lim[w]) || (cmask[w] & (x[w] | z[w]))) return SPS_ERR_ARG;
  if ((x[0] | x[1] | z[0] | z[1]) == 0) return SPS_ERR_ARG;
  const sps_status fs = flush_reset(s);
  if (fs != SPS_OK) return fs;
  if ((x[0] | x[1]) == 0) {
    // A string of Z factors is diagonal: exp(-i t/2 P) multiplies a label by
    // e^(-i t/2) or e^(i t/2) as the parity of its z bits is 0 or 1. A ladder of
    // CNOTs puts that parity on the top z qubit, Rz(t) applies the phase, the
    // ladder is undone: one fused run.
    std::vector<uint32_t> bits;
    for (uint32_t q = 0; q < s->nqubits; ++q)
      if ((z[q >> 6] >> (q & 63)) & 1ull) bits.push_back(q);
    const uint32_t t = bits.back();
    std::vector<sps_gate> g;
    auto rec = [&](uint8_t op, uint32_t tq, const uint64_t c[2], double th) {
      sps_gate r;
      std::memset(&r, 0, sizeof(r));
      r.op = op;
      r.t0 = (uint16_t)tq;
      r.cmask[0] = c[0];
      r.cmask[1] = c[1];
      r.theta = th;
      g.push_back(r);
    };
    for (size_t i = 0; i + 1 < bits.size(); ++i) {
      const uint64_t c[2] = {bits[i] < 64 ? 1ull << bits[i] : 0ull,
                             bits[i] >= 64 ? 1ull << (bits[i] - 64) : 0ull};
      rec(SPS_OP_X, t, c, 0.0);
    }
    rec(SPS_OP_RZ, t, cmask, theta);
    for (size_t i = bits.size() - 1; i-- > 0;) {
      const uint64_t c[2] = {bits[i] < 64 ? 1ull << bits[i] : 0ull,
                             bits[i] >= 64 ? 1ull << (bits[i] - 64) : 0ull};
      rec(SPS_OP_X, t, c, 0.0);
    }
    return sps_apply(s, g.data(), g.size(), prune_eps, nullptr);
  }
  BranchOp op;
  std::memset(&op, 0, sizeof(op));
  op.c[0] = cmask[0];
  op.c[1] = cmask[1];
  op.m[0] = x[0];
  op.m[1] = x[1];
  op.sbit = x[0] ? (uint32_t)__builtin_ctzll(x[0]) : 64u + (uint32_t)__builtin_ctzll(x[1]);
  op.pauli = 1;
  op.pz[0] = z[0];
  op.pz[1] = z[1];
  op.ny = (uint32_t)(__builtin_popcountll(x[0] & z[0]) + __builtin_popcountll(x[1] & z[1])) & 3u;
  op.m_re[0][0] = op.m_re[1][1] = std::cos(0.5 * theta);
  op.psin = std::sin(0.5 * theta);
  op.real_m = 0;
  // knowledge: the flipped qubits vary afterwards unless a control is known 0
  const bool never = ((cmask[0] & s->kb.known[0] & ~s->kb.val[0]) |
                      (cmask[1] & s->kb.known[1] & ~s->kb.val[1])) != 0ull;
  if (!never) {
    s->kb.known[0] &= ~x[0];
    s->kb.known[1] &= ~x[1];
  }
  const LaunchCfg lc = cfg_of(s);
  ++s->apply_serial;
  const uint32_t serial = ++s->pass_serial;
  const uint64_t tag = (uint64_t)s->apply_serial << 32;
  s->amp_force = true;   // an out-of-place pass: labels move, index slots are taken
  const sps_status bs = launch_branch_pass(s, lc, op, prune_eps, serial, tag, probe_limit_of(s));
  if (bs != SPS_OK) return bs;
  s->counters.gates += 1;
  return SPS_OK;
}

sps_status sps_measure(sps_state* s, uint32_t qubit, double r, double* out) {
  if (!s || !out || qubit >= s->nqubits || !(r >= 0.0 && r < 1.0)) return SPS_ERR_ARG;
  ++s->version;
  const sps_status fs = flush_reset(s);
  if (fs != SPS_OK) return fs;
  const LaunchCfg lc = cfg_of(s);
  const uint32_t serial = ++s->pass_serial;
  s->amp_force = true;   // the collapse moves labels
  ProfScope ps(s, 8, serial, 1, 1u);
  const int n = launch_measure(lc, s->kw, s->ctl, s->bufs, qubit, r, s->partials, s->prob_blocks,
                               s->dmeasure, s->nnz_bound, s->masks.writer(), ps.slot);
  ps.done();
  if (n < 0) return cuda_ok(cudaGetLastError());
  s->counters.kernel_launches += (uint64_t)n;
  s->counters.gates += 1;
  if (cudaMemcpyAsync(out, s->dmeasure, 2 * sizeof(double), cudaMemcpyDefault, s->stream) !=
      cudaSuccess)
    return cuda_ok(cudaGetLastError());
  return SPS_OK;
}

sps_status sps_set_option(sps_state* s, sps_option opt, int64_t v) {
  if (!s) return SPS_ERR_ARG;
  switch (opt) {
    case SPS_OPT_LOAD_FACTOR_PCT:
      if (v < 10 || v > 90) return SPS_ERR_ARG;
      s->load_pct = (uint32_t)v;
      return SPS_OK;
    case SPS_OPT_PROBE_LIMIT:
      if (v < 0 || v > 0xFFFFFFFFll) return SPS_ERR_ARG;
      s->probe_limit = (uint32_t)v;
      return SPS_OK;
    case SPS_OPT_BLOCK_THREADS:
      if (v != 128 && v != 256) return SPS_ERR_ARG;
      s->threads = (int)v;
      return SPS_OK;
    case SPS_OPT_MAX_FUSED_OPS:
      if (v < 1 || v > (int64_t)kMaxFusedOps) return SPS_ERR_ARG;
      s->max_fused_ops = (uint32_t)v;
      return SPS_OK;
    case SPS_OPT_BITSLICE_GROUPS:
      if (v < 0 || v > 32 || (v & 1)) return SPS_ERR_ARG;
      s->bs_groups = (uint32_t)v;
      return SPS_OK;
    case SPS_OPT_EXPAND:
      if (v != 0 && v != 1) return SPS_ERR_ARG;
      s->expand = v == 1;
      return SPS_OK;
    case SPS_OPT_FOLD:
      if (v != 0 && v != 1) return SPS_ERR_ARG;
      s->fold = v == 1;
      return SPS_OK;
    case SPS_OPT_COMMUTE:
      if (v != 0 && v != 1) return SPS_ERR_ARG;
      s->commute = v == 1;
      return SPS_OK;
    case SPS_OPT_LAYER_GATES:
      if (v < 1 || v > (int64_t)kMaxLayerGates) return SPS_ERR_ARG;
      s->layer_max = (uint32_t)v;
      return SPS_OK;
    case SPS_OPT_EXPAND_WALK:
      if (v != 0 && v != 1) return SPS_ERR_ARG;
      s->expand_walk = v == 1;
      return SPS_OK;
    case SPS_OPT_AMP_ONLY:
      if (v != 0 && v != 1) return SPS_ERR_ARG;
      s->amp = v == 1;
      return SPS_OK;
    case SPS_OPT_BITSLICE_JIT:
      if (v < 0 || v > 2) return SPS_ERR_ARG;
      s->bs_jit = (int)v;
      return SPS_OK;
    case SPS_OPT_PLAN_CACHE:
      if (v != 0 && v != 1) return SPS_ERR_ARG;
      s->plan_cache = v == 1;
      return SPS_OK;
    case SPS_OPT_FALLBACK_CHAIN:
      if (v != 0 && v != 1) return SPS_ERR_ARG;
      s->chain = v == 1;
      return SPS_OK;
    case SPS_OPT_READOUT_MIN_PLANES:
      if (v < 0 || v > 128) return SPS_ERR_ARG;
      s->rd_min_planes = (uint32_t)v;
      return SPS_OK;
    case SPS_OPT_FUSED_LABELS:
      if (v != 0 && v != 1 && v != 2 && v != 4 && v != 8) return SPS_ERR_ARG;
      s->fused_labels = (int)v;
      return SPS_OK;
    case SPS_OPT_BRANCH_FORM:
      if (v < 0 || v > 2) return SPS_ERR_ARG;
      s->branch_form = (int)v;
      return SPS_OK;
    case SPS_OPT_SMALL_RUN_CAP:
      if (v < 0 || v > (int64_t)kSmallCap) return SPS_ERR_ARG;
      s->small_cap = (uint32_t)v;
      return SPS_OK;
    case SPS_OPT_BITSLICE_MIN_OPS:
      if (v < 0 || v > 1000000) return SPS_ERR_ARG;
      s->bitslice_min_ops = (uint32_t)v;
      return SPS_OK;
    case SPS_OPT_BITSLICE_MIN_NNZ:
      if (v < 0) return SPS_ERR_ARG;
      s->bitslice_min_nnz = (uint64_t)v;
      return SPS_OK;
    case SPS_OPT_PROFILE:
      if (v != 0 && v != 1) return SPS_ERR_ARG;
      s->profile = v == 1;
      return SPS_OK;
    case SPS_OPT_COOP_WIDTH:
      if (v != 1 && v != 2 && v != 4 && v != 8) return SPS_ERR_ARG;
      s->coop = (int)v;
      return SPS_OK;
  }
  return SPS_ERR_ARG;
}

// ---- autotuner of the plain path --------------------------------------------------
// Options that shape how the path runs but not what it computes, plus the
// fusion length, chosen per size class (label width, log2 of the projected
// peak nonzeros) by timing whole steps; the choice can be kept in a text file,
// one line per class: "sps-tune 1 kw=K log2peak=P load_factor_pct=.. ...".
static bool tune_choice_ok(const sps_tune_choice& c) {
  return c.load_factor_pct >= 10 && c.load_factor_pct <= 90 && c.bitslice_groups <= 32 &&
         (c.bitslice_groups & 1u) == 0 &&
         (c.fused_labels == 0 || c.fused_labels == 1 || c.fused_labels == 2 ||
          c.fused_labels == 4 || c.fused_labels == 8) &&
         c.max_fused_ops >= 1 && c.max_fused_ops <= kMaxFusedOps;
}

sps_status sps_tune_cache_lookup(const char* path, uint32_t kw, uint32_t log2peak,
                                 sps_tune_choice* out) {
  if (!path || !out || (kw != 1 && kw != 2)) return SPS_ERR_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return SPS_ERR_ARG;
  char line[512];
  bool found = false;
  sps_tune_choice best;
  std::memset(&best, 0, sizeof(best));
  while (std::fgets(line, sizeof(line), f)) {
    sps_tune_choice c;
    std::memset(&c, 0, sizeof(c));
    float ms = 0.f;
    if (std::sscanf(line,
                    "sps-tune 1 kw=%u log2peak=%u load_factor_pct=%u bitslice_groups=%u "
                    "fused_labels=%u max_fused_ops=%u ms=%f",
                    &c.kw, &c.log2peak, &c.load_factor_pct, &c.bitslice_groups, &c.fused_labels,
                    &c.max_fused_ops, &ms) != 7)
      continue;
    if (c.kw != kw || c.log2peak != log2peak || !tune_choice_ok(c)) continue;
    c.ms = ms;
    c.from_cache = 1;
    best = c;   // a later line of the class replaces an earlier one
    found = true;
  }
  std::fclose(f);
  if (!found) return SPS_ERR_ARG;
  *out = best;
  return SPS_OK;
}

static void tune_set(sps_state* s, const sps_tune_choice& c) {
  s->load_pct = c.load_factor_pct;
  s->bs_groups = c.bitslice_groups;
  s->fused_labels = (int)c.fused_labels;
  s->max_fused_ops = c.max_fused_ops;
}

// Mean wall time of `repeats` whole steps (reset, apply, sync) under choice c,
// after one untimed step that compiles and uploads the plan for it.
static sps_status tune_time(sps_state* s, const sps_gate* gates, size_t ngates, double eps,
                            uint32_t repeats, const sps_tune_choice& c, float* ms) {
  tune_set(s, c);
  double total = 0.0;
  for (uint32_t r = 0; r <= repeats; ++r) {
    const auto t0 = std::chrono::steady_clock::now();
    sps_status st = sps_reset(s);
    if (st == SPS_OK) st = sps_apply(s, gates, ngates, eps, nullptr);
    if (st == SPS_OK) st = sps_sync(s, nullptr);
    if (st != SPS_OK) return st;
    const auto t1 = std::chrono::steady_clock::now();
    if (r > 0) total += std::chrono::duration<double, std::milli>(t1 - t0).count();
  }
  *ms = (float)(total / repeats);
  return SPS_OK;
}

sps_status sps_tune(sps_state* s, const sps_gate* gates, size_t ngates, double prune_eps,
                    uint32_t repeats, const char* cache_path, sps_tune_choice* out) {
  if (!s || !out || (ngates && !gates) || !(prune_eps >= 0.0) || repeats < 1 || repeats > 1000)
    return SPS_ERR_ARG;
  std::vector<Pass> passes;
  size_t bad = 0;
  const sps_status cs = compile(gates, ngates, s->nqubits, 0, &passes, &bad);
  if (cs != SPS_OK) return cs;
  const uint64_t peak = projected_peak(passes, s->capacity);
  uint32_t lg = 0;
  while (lg < 63 && (1ull << lg) < peak) ++lg;
  const uint32_t kw = (uint32_t)s->kw;
  if (cache_path) {
    sps_tune_choice c;
    if (sps_tune_cache_lookup(cache_path, kw, lg, &c) == SPS_OK) {
      tune_set(s, c);
      const sps_status rs = sps_reset(s);
      if (rs != SPS_OK) return rs;
      *out = c;
      return SPS_OK;
    }
  }
  sps_tune_choice best;
  std::memset(&best, 0, sizeof(best));
  best.kw = kw;
  best.log2peak = lg;
  best.load_factor_pct = s->load_pct;
  best.bitslice_groups = s->bs_groups;
  best.fused_labels = (uint32_t)s->fused_labels;
  best.max_fused_ops = s->max_fused_ops;
  sps_status st = tune_time(s, gates, ngates, prune_eps, repeats, best, &best.ms);
  if (st != SPS_OK) return st;
  // one option at a time, from the best so far
  static const uint32_t kLoad[] = {30, 50, 70};
  static const uint32_t kGroups[] = {0, 8, 16, 32};
  static const uint32_t kLabels[] = {0, 2, 4, 8};
  static const uint32_t kFused[] = {128, 256, 512};
  for (int dim = 0; dim < 4; ++dim) {
    const uint32_t* vals = dim == 0 ? kLoad : dim == 1 ? kGroups : dim == 2 ? kLabels : kFused;
    const int nv = dim == 0 || dim == 3 ? 3 : 4;
    const sps_tune_choice base = best;
    for (int k = 0; k < nv; ++k) {
      sps_tune_choice c = base;
      uint32_t* field = dim == 0 ? &c.load_factor_pct : dim == 1 ? &c.bitslice_groups
                        : dim == 2 ? &c.fused_labels : &c.max_fused_ops;
      if (*field == vals[k]) continue;
      *field = vals[k];
      if (!tune_choice_ok(c)) continue;
      st = tune_time(s, gates, ngates, prune_eps, repeats, c, &c.ms);
      if (st != SPS_OK) return st;
      if (c.ms < best.ms) best = c;
    }
  }
  tune_set(s, best);
  st = sps_reset(s);
  if (st != SPS_OK) return st;
  if (cache_path) {
    FILE* f = std::fopen(cache_path, "a");
    if (f) {
      std::fprintf(f,
                   "sps-tune 1 kw=%u log2peak=%u load_factor_pct=%u bitslice_groups=%u "
                   "fused_labels=%u max_fused_ops=%u ms=%.4f\n",
                   best.kw, best.log2peak, best.load_factor_pct, best.bitslice_groups,
                   best.fused_labels, best.max_fused_ops, best.ms);
      std::fclose(f);
    }
  }
  best.from_cache = 0;
  *out = best;
  return SPS_OK;
}

sps_status sps_barrier_selftest(uint32_t skip_block, uint32_t spins, sps_status* result) {
  if (!result || spins < 1) return SPS_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SPS_ERR_NO_DEVICE;
  }
  int st = 0;
  if (barrier_selftest(skip_block, spins, &st) < 0) return SPS_ERR_CUDA;
  *result = (sps_status)st;
  return SPS_OK;
}

sps_status sps_get_counters(sps_state* s, sps_counters* out) {
  if (!s || !out) return SPS_ERR_ARG;
  *out = s->counters;
  return SPS_OK;
}

sps_status sps_plan(const sps_gate* gates, size_t ngates, uint32_t nqubits, uint32_t max_fused_ops,
                    uint32_t* kind, uint64_t* first_gate, uint32_t* ops, size_t cap,
                    size_t* npasses, size_t* failed_gate) {
  if ((ngates && !gates) || !npasses || nqubits < 1 || nqubits > 127) return SPS_ERR_ARG;
  std::vector<Pass> passes;
  size_t bad = 0;
  const sps_status st = compile(gates, ngates, nqubits, max_fused_ops, &passes, &bad);
  if (st != SPS_OK) {
    if (failed_gate) *failed_gate = bad;
    return st;
  }
  *npasses = passes.size();
  for (size_t i = 0; i < passes.size() && i < cap; ++i) {
    if (kind) kind[i] = passes[i].kind;
    if (first_gate) first_gate[i] = passes[i].first_gate;
    if (ops) ops[i] = passes[i].kind == PASS_FUSED ? (uint32_t)passes[i].ops.size() : 1u;
  }
  return SPS_OK;
}

sps_status sps_commute(const sps_gate* gates, size_t ngates, uint32_t nqubits, sps_gate* out,
                       size_t cap, size_t* nout, size_t* failed_gate) {
  if ((ngates && !gates) || !nout || (cap && !out) || nqubits < 1 || nqubits > 127)
    return SPS_ERR_ARG;
  std::vector<sps_gate> g;
  std::vector<size_t> origin;
  size_t bad = 0;
  const sps_status st = commute_gates(gates, ngates, nqubits, &g, &origin, &bad);
  if (st != SPS_OK) {
    if (failed_gate) *failed_gate = bad;
    return st;
  }
  *nout = g.size();
  if (g.size() > cap) return SPS_ERR_CAPACITY;
  if (!g.empty()) std::memcpy(out, g.data(), g.size() * sizeof(sps_gate));
  return SPS_OK;
}

}  // extern "C"
