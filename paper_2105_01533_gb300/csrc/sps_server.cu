// Serving loop: continuous batching of circuit requests.
//
// Requests are admitted in arrival order while an active slot and enough of the
// device-memory budget (their projected peak state) are free. Each tick
// advances every active request by at most `passes_per_tick` passes:
//   * small requests (capacity <= kServeSmallCap) together in one batched launch
//     (k_batch) on the server's stream, each state resident on the device
//     between ticks;
//   * large requests each as a whole-GPU state (sps_state) on its own stream,
//     one sps_apply of the next passes' gates per tick,
// so requests of both kinds run concurrently on the device. A finished
// request's state is copied to the host and its device memory released before
// the next tick admits new requests.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "sps.h"
#include "sps_batch.h"
#include "sps_internal.h"

using namespace sps;

namespace {

constexpr uint64_t kServeSmallCap = 1u << 16;

enum ReqState : int { REQ_PENDING = 0, REQ_ACTIVE = 1, REQ_DONE = 2 };

struct Request {
  uint64_t id = 0;
  uint32_t nqubits = 0;
  uint64_t capacity = 0;
  double eps = 0.0;
  std::vector<sps_gate> gates;
  std::vector<Pass> passes;
  int state = REQ_PENDING;
  sps_status status = SPS_OK;
  size_t failed_gate = 0;
  uint64_t submit_tick = 0, admit_tick = 0, done_tick = 0;
  bool small = true;
  uint64_t mem = 0;        // budget charged
  uint64_t work = 0;
  // small route
  int slot = -1;
  void* plan = nullptr;
  size_t plan_bytes = 0;
  void* buf = nullptr;
  size_t buf_bytes = 0;
  // large route
  sps_state* st = nullptr;
  cudaStream_t stream = nullptr;
  size_t next_pass = 0;
  // result
  std::vector<uint64_t> hi, lo;
  std::vector<double> re, im;
  uint64_t updates = 0;
};

}  // namespace

struct sps_server {
  cudaStream_t stream = nullptr;
  int device = 0, sms = 0;
  uint64_t budget = 0, used = 0;
  uint32_t max_active = 0, passes_per_tick = 0;
  uint64_t tick = 0, next_id = 1;
  BatchConfig cfg{512, 2, 1024, 0};
  std::map<uint64_t, Request> reqs;
  std::deque<uint64_t> pending;
  std::vector<uint64_t> active;
  std::vector<uint64_t> last_done;   // finished in the last tick
  // small-route device state: descriptors per slot
  BatchDesc* desc = nullptr;
  std::vector<BatchDesc> host_desc;
  std::vector<int> slot_free;
  uint32_t* order = nullptr;
  uint32_t* head = nullptr;
  uint32_t* gtabs = nullptr;
  uint32_t gtab_slots = 0;
  uint64_t launches = 0;
};

namespace {

sps_status cst(cudaError_t e) {
  if (e == cudaSuccess) return SPS_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? SPS_ERR_OOM : SPS_ERR_CUDA;
}

void release_request(sps_server* s, Request& r) {
  if (r.small) {
    if (r.buf) hook_free(r.buf, r.buf_bytes, s->stream);
    if (r.plan) hook_free(r.plan, r.plan_bytes, s->stream);
    r.buf = r.plan = nullptr;
    if (r.slot >= 0) s->slot_free.push_back(r.slot);
    r.slot = -1;
  } else {
    if (r.st) sps_destroy(r.st);
    r.st = nullptr;
    if (r.stream) cudaStreamDestroy(r.stream);
    r.stream = nullptr;
  }
  s->used -= r.mem;
  r.mem = 0;
}

// bytes a request holds while active
uint64_t request_bytes(const Request& r, size_t plan_bytes) {
  if (r.small) return 64 * r.capacity + plan_bytes;
  // two label/amplitude buffers, the gather index table, arenas (rough)
  return 64 * r.capacity + 32 * r.capacity + (4u << 20);
}

sps_status admit(sps_server* s, Request& r) {
  sps_status st = SPS_OK;
  if (r.small) {
    std::vector<unsigned char> blob;
    uint32_t pass_off = 0;
    pack_circuit(r.passes, r.eps, &blob, &pass_off, &r.work, r.capacity);
    r.plan_bytes = std::max<size_t>(blob.size(), 16);
    r.buf_bytes = 64 * r.capacity;
    r.plan = hook_alloc(r.plan_bytes, s->stream);
    r.buf = r.plan ? hook_alloc(r.buf_bytes, s->stream) : nullptr;
    if (!r.plan || !r.buf) {
      release_request(s, r);
      return SPS_ERR_OOM;
    }
    if (!blob.empty() &&
        (st = cst(cudaMemcpyAsync(r.plan, blob.data(), blob.size(), cudaMemcpyHostToDevice,
                                  s->stream))) != SPS_OK)
      return st;
    r.slot = s->slot_free.back();
    s->slot_free.pop_back();
    BatchDesc d;
    std::memset(&d, 0, sizeof(d));
    unsigned char* base = static_cast<unsigned char*>(r.buf);
    const size_t cap = r.capacity;
    for (int k = 0; k < 2; ++k) {
      unsigned char* bb = base + (size_t)k * 32 * cap;
      d.lo[k] = reinterpret_cast<uint64_t*>(bb);
      d.hi[k] = reinterpret_cast<uint64_t*>(bb + 8 * cap);
      d.re[k] = reinterpret_cast<double*>(bb + 16 * cap);
      d.im[k] = reinterpret_cast<double*>(bb + 24 * cap);
    }
    d.plan = static_cast<const unsigned char*>(r.plan);
    d.pass_off = pass_off;
    d.npasses = (uint32_t)r.passes.size();
    d.kw = r.nqubits <= 63 ? 1u : 2u;
    d.capacity = r.capacity;
    s->host_desc[r.slot] = d;
    if ((st = cst(cudaMemcpyAsync(s->desc + r.slot, &s->host_desc[r.slot], sizeof(BatchDesc),
                                  cudaMemcpyHostToDevice, s->stream))) != SPS_OK)
      return st;
    if (launch_batch_reset(s->stream, s->desc + r.slot, 1) < 0) return cst(cudaGetLastError());
  } else {
    if ((st = cst(cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking))) != SPS_OK) return st;
    if ((st = sps_create(r.nqubits, r.capacity, r.stream, &r.st)) != SPS_OK) {
      release_request(s, r);
      return st;
    }
    // a request's passes reach the state a tick at a time, so its long runs
    // are compiled per slice: the general bit-sliced kernel, not one compiled
    // at run time for each run (a compile costs more than most requests)
    if ((st = sps_set_option(r.st, SPS_OPT_BITSLICE_JIT, 0)) != SPS_OK) {
      release_request(s, r);
      return st;
    }
    r.next_pass = 0;
  }
  return SPS_OK;
}

// copies a finished request's state to the host
sps_status harvest(sps_server* s, Request& r) {
  uint64_t n = 0;
  if (r.small) {
    const BatchDesc& d = s->host_desc[r.slot];
    n = d.nnz;
    const unsigned c = d.cur;
    r.lo.resize(n);
    r.hi.resize(n);
    r.re.resize(n);
    r.im.resize(n);
    r.updates = d.updates;
    if (n) {
      bool ok = cudaMemcpyAsync(r.lo.data(), d.lo[c], 8 * n, cudaMemcpyDeviceToHost, s->stream) ==
                    cudaSuccess &&
                cudaMemcpyAsync(r.hi.data(), d.hi[c], 8 * n, cudaMemcpyDeviceToHost, s->stream) ==
                    cudaSuccess &&
                cudaMemcpyAsync(r.re.data(), d.re[c], 8 * n, cudaMemcpyDeviceToHost, s->stream) ==
                    cudaSuccess &&
                cudaMemcpyAsync(r.im.data(), d.im[c], 8 * n, cudaMemcpyDeviceToHost, s->stream) ==
                    cudaSuccess;
      if (!ok) return cst(cudaGetLastError());
      const sps_status st = cst(cudaStreamSynchronize(s->stream));
      if (st != SPS_OK) return st;
    }
    if (d.kw == 1) std::fill(r.hi.begin(), r.hi.end(), 0ull);
  } else {
    sps_status st = sps_nnz(r.st, &n);
    if (st != SPS_OK) return st;
    if ((st = sps_get_updates(r.st, &r.updates)) != SPS_OK) return st;
    r.lo.resize(n);
    r.hi.resize(n);
    r.re.resize(n);
    r.im.resize(n);
    uint64_t got = 0;
    if (n && (st = sps_get_amplitudes(r.st, r.hi.data(), r.lo.data(), r.re.data(), r.im.data(), n,
                                      &got)) != SPS_OK)
      return st;
  }
  return SPS_OK;
}

}  // namespace

extern "C" {

sps_status sps_server_create(uint64_t mem_budget_bytes, uint32_t max_active,
                             uint32_t passes_per_tick, void* cuda_stream, sps_server** out) {
  if (!out || max_active < 1 || max_active > 65536 || mem_budget_bytes == 0) return SPS_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return SPS_ERR_NO_DEVICE;
  }
  sps_server* s = new (std::nothrow) sps_server;
  if (!s) return SPS_ERR_OOM;
  s->stream = (cudaStream_t)cuda_stream;
  s->budget = mem_budget_bytes;
  s->max_active = max_active;
  s->passes_per_tick = passes_per_tick;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return SPS_ERR_CUDA;
  }
  uint32_t slots = 256;
  while (slots < 4 * kServeSmallCap) slots <<= 1;
  s->gtab_slots = slots;
  const size_t blocks = (size_t)s->sms * s->cfg.blocks_per_sm;
  s->desc = static_cast<BatchDesc*>(hook_alloc(sizeof(BatchDesc) * max_active, s->stream));
  s->order = static_cast<uint32_t*>(hook_alloc(sizeof(uint32_t) * max_active, s->stream));
  s->head = static_cast<uint32_t*>(hook_alloc(256, s->stream));
  s->gtabs = static_cast<uint32_t*>(hook_alloc(sizeof(uint32_t) * slots * blocks, s->stream));
  if (!s->desc || !s->order || !s->head || !s->gtabs) {
    sps_server_destroy(s);
    return SPS_ERR_OOM;
  }
  s->host_desc.assign(max_active, BatchDesc());
  for (int i = (int)max_active - 1; i >= 0; --i) s->slot_free.push_back(i);
  *out = s;
  return SPS_OK;
}

void sps_server_destroy(sps_server* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  for (auto& kv : s->reqs)
    if (kv.second.state == REQ_ACTIVE) release_request(s, kv.second);
  const size_t blocks = (size_t)s->sms * s->cfg.blocks_per_sm;
  if (s->desc) hook_free(s->desc, sizeof(BatchDesc) * s->max_active, s->stream);
  if (s->order) hook_free(s->order, sizeof(uint32_t) * s->max_active, s->stream);
  if (s->head) hook_free(s->head, 256, s->stream);
  if (s->gtabs) hook_free(s->gtabs, sizeof(uint32_t) * s->gtab_slots * blocks, s->stream);
  cudaStreamSynchronize(s->stream);
  cudaGetLastError();
  delete s;
}

sps_status sps_server_submit(sps_server* s, uint32_t nqubits, uint64_t capacity,
                             const sps_gate* gates, size_t ngates, double prune_eps, uint64_t* id,
                             size_t* failed_gate) {
  if (!s || !id || nqubits < 1 || nqubits > 127 || capacity < 1 || capacity > (1ull << 32) ||
      (ngates && !gates) || !(prune_eps >= 0.0))
    return SPS_ERR_ARG;
  Request r;
  r.nqubits = nqubits;
  r.capacity = capacity;
  r.eps = prune_eps;
  size_t bad = 0;
  const sps_status st = compile(gates, ngates, nqubits, 0, &r.passes, &bad);
  if (st != SPS_OK) {
    if (failed_gate) *failed_gate = bad;
    return st;
  }
  r.gates.assign(gates, gates + ngates);
  // the state is sized (and the request charged) for its projected peak
  r.capacity = projected_peak(r.passes, capacity);
  r.small = r.capacity <= kServeSmallCap;
  r.id = s->next_id++;
  r.submit_tick = s->tick;
  if (request_bytes(r, 0) > s->budget) return SPS_ERR_CAPACITY;   // could never be admitted
  *id = r.id;
  s->pending.push_back(r.id);
  s->reqs.emplace(r.id, std::move(r));
  return SPS_OK;
}

sps_status sps_server_tick(sps_server* s, uint32_t* n_active, uint32_t* n_pending,
                           uint32_t* n_done) {
  if (!s) return SPS_ERR_ARG;
  ++s->tick;
  sps_status st = SPS_OK;
  // 1. admission, in arrival order, while a slot and the budget allow
  while (!s->pending.empty() && s->active.size() < s->max_active) {
    Request& r = s->reqs[s->pending.front()];
    const uint64_t need = request_bytes(r, 64 * 1024);
    if (s->used + need > s->budget) break;
    if (r.small && s->slot_free.empty()) break;
    r.mem = need;
    s->used += need;
    if ((st = admit(s, r)) != SPS_OK) {
      if (st == SPS_ERR_OOM) break;   // retry on a later tick
      return st;
    }
    r.state = REQ_ACTIVE;
    r.admit_tick = s->tick;
    s->active.push_back(r.id);
    s->pending.pop_front();
  }
  // 2. one step for every active request
  std::vector<uint32_t> small_slots;
  std::vector<std::pair<uint64_t, uint32_t>> by_work;
  for (uint64_t id : s->active) {
    Request& r = s->reqs[id];
    if (r.small) {
      by_work.push_back({r.work, (uint32_t)r.slot});
    } else {
      const size_t p0 = r.next_pass;
      size_t p1 = s->passes_per_tick ? std::min(r.passes.size(), p0 + s->passes_per_tick)
                                     : r.passes.size();
      const size_t g0 = p0 < r.passes.size() ? r.passes[p0].first_gate : r.gates.size();
      const size_t g1 = p1 < r.passes.size() ? r.passes[p1].first_gate : r.gates.size();
      if (g1 > g0 && (st = sps_apply(r.st, r.gates.data() + g0, g1 - g0, r.eps, nullptr)) != SPS_OK)
        return st;
      r.next_pass = p1;
    }
  }
  if (!by_work.empty()) {
    std::sort(by_work.begin(), by_work.end(), [](auto& a, auto& b) { return a.first > b.first; });
    for (auto& w : by_work) small_slots.push_back(w.second);
    if ((st = cst(cudaMemcpyAsync(s->order, small_slots.data(), sizeof(uint32_t) * small_slots.size(),
                                  cudaMemcpyHostToDevice, s->stream))) != SPS_OK ||
        (st = cst(cudaMemsetAsync(s->head, 0, sizeof(uint32_t), s->stream))) != SPS_OK)
      return st;
    if (launch_batch(s->stream, s->sms, s->cfg, s->desc, s->order, (uint32_t)small_slots.size(),
                     s->head, s->gtabs, s->gtab_slots, s->passes_per_tick) < 0)
      return cst(cudaGetLastError());
    ++s->launches;
    // read back every descriptor (small, and the copy is stream ordered)
    if ((st = cst(cudaMemcpyAsync(s->host_desc.data(), s->desc, sizeof(BatchDesc) * s->max_active,
                                  cudaMemcpyDeviceToHost, s->stream))) != SPS_OK)
      return st;
  }
  if ((st = cst(cudaStreamSynchronize(s->stream))) != SPS_OK) return st;
  // 3. harvest finished requests
  uint32_t done = 0;
  std::vector<uint64_t> still;
  s->last_done.clear();
  for (uint64_t id : s->active) {
    Request& r = s->reqs[id];
    bool finished = false;
    if (r.small) {
      const BatchDesc& d = s->host_desc[r.slot];
      if (d.status != 0) {
        r.status = (sps_status)d.status;
        r.failed_gate = d.failed_pass < r.passes.size() ? r.passes[d.failed_pass].first_gate : 0;
        finished = true;
      } else if (d.next_pass >= d.npasses) {
        finished = true;
      }
    } else {
      size_t fg = 0;
      const sps_status ss = sps_sync(r.st, &fg);
      if (ss != SPS_OK) {
        r.status = ss;
        r.failed_gate = fg;
        finished = true;
      } else if (r.next_pass >= r.passes.size()) {
        finished = true;
      }
    }
    if (!finished) {
      still.push_back(id);
      continue;
    }
    if ((st = harvest(s, r)) != SPS_OK) return st;
    release_request(s, r);
    r.state = REQ_DONE;
    r.done_tick = s->tick;
    s->last_done.push_back(r.id);
    ++done;
  }
  s->active.swap(still);
  if (n_active) *n_active = (uint32_t)s->active.size();
  if (n_pending) *n_pending = (uint32_t)s->pending.size();
  if (n_done) *n_done = done;
  return SPS_OK;
}

sps_status sps_server_poll(sps_server* s, uint64_t id, sps_server_request_info* info) {
  if (!s || !info) return SPS_ERR_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return SPS_ERR_ARG;
  const Request& r = it->second;
  info->state = r.state;
  info->status = r.status;
  info->failed_gate = r.failed_gate;
  info->nnz = r.state == REQ_DONE ? r.lo.size() : 0;
  info->submit_tick = r.submit_tick;
  info->admit_tick = r.admit_tick;
  info->done_tick = r.done_tick;
  info->large = r.small ? 0 : 1;
  info->updates = r.updates;
  return SPS_OK;
}

sps_status sps_server_result(sps_server* s, uint64_t id, uint64_t* key_hi, uint64_t* key_lo,
                             double* re, double* im, uint64_t cap, uint64_t* nnz_out) {
  if (!s || !key_lo || !re || !im || !nnz_out) return SPS_ERR_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second.state != REQ_DONE) return SPS_ERR_ARG;
  Request& r = it->second;
  *nnz_out = r.lo.size();
  if (r.lo.size() > cap) return SPS_ERR_CAPACITY;
  const size_t n = r.lo.size();
  std::memcpy(key_lo, r.lo.data(), 8 * n);
  std::memcpy(re, r.re.data(), 8 * n);
  std::memcpy(im, r.im.data(), 8 * n);
  if (key_hi) std::memcpy(key_hi, r.hi.data(), 8 * n);
  s->reqs.erase(it);   // the result is handed over once
  return SPS_OK;
}

sps_status sps_server_completed(sps_server* s, uint64_t* ids, size_t cap, size_t* n) {
  if (!s || !n || (cap && !ids)) return SPS_ERR_ARG;
  *n = s->last_done.size();
  for (size_t i = 0; i < s->last_done.size() && i < cap; ++i) ids[i] = s->last_done[i];
  return s->last_done.size() > cap ? SPS_ERR_CAPACITY : SPS_OK;
}

sps_status sps_server_stats(sps_server* s, uint64_t* ticks, uint64_t* launches, uint64_t* bytes_in_use) {
  if (!s) return SPS_ERR_ARG;
  if (ticks) *ticks = s->tick;
  if (launches) *launches = s->launches;
  if (bytes_in_use) *bytes_in_use = s->used;
  return SPS_OK;
}

}  // extern "C"
