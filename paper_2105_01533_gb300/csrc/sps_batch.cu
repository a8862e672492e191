// Batched execution: many independent circuits in one persistent launch.
//
// Every circuit is described by a BatchDesc (its two state buffers, its
// compiled passes and its progress). The grid is persistent (a fixed number of
// blocks per SM); each block takes the next circuit from a queue ordered by
// estimated work, largest first, and runs up to `max_passes` of its passes with
// the CTA engine (sps_cta_engine.cuh): in shared memory when the circuit's
// capacity fits, else on the circuit's own global buffers with a per-block
// index table. Progress, nonzero count and status go back to the descriptor, so
// a circuit can be resumed by a later launch (the serving loop does that).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "sps.h"
#include "sps_batch.h"
#include "sps_cta_engine.cuh"
#include "sps_internal.h"

namespace sps {
namespace {

using namespace dev;

__device__ __forceinline__ cta::Bufs desc_bufs(const BatchDesc& d, unsigned which) {
  cta::Bufs b;
  b.lo = which ? d.lo[1] : d.lo[0];
  b.hi = which ? d.hi[1] : d.hi[0];
  b.re = which ? d.re[1] : d.re[0];
  b.im = which ? d.im[1] : d.im[0];
  return b;
}

template <int KW>
__device__ void run_circuit(BatchDesc* dp, uint32_t max_passes, uint32_t smem_cap,
                            unsigned char* smem, uint32_t* gtab, uint32_t gtab_slots,
                            uint32_t* warp_sums) {
  const BatchDesc d = *dp;
  const uint32_t p0 = d.next_pass;
  uint32_t p1 = d.npasses;
  if (max_passes && p0 + max_passes < p1) p1 = p0 + max_passes;
  const RunPass* passes = reinterpret_cast<const RunPass*>(d.plan + d.pass_off);
  uint32_t n = (uint32_t)d.nnz;
  unsigned cur = d.cur;
  uint32_t done;
  uint64_t upd = 0;
  if (d.capacity <= smem_cap) {
    cta::Bufs A, B;
    A.lo = reinterpret_cast<uint64_t*>(smem);
    A.hi = A.lo + smem_cap;
    A.re = reinterpret_cast<double*>(A.hi + smem_cap);
    A.im = A.re + smem_cap;
    B.lo = reinterpret_cast<uint64_t*>(A.im + smem_cap);
    B.hi = B.lo + smem_cap;
    B.re = reinterpret_cast<double*>(B.hi + smem_cap);
    B.im = B.re + smem_cap;
    uint32_t* stab = reinterpret_cast<uint32_t*>(B.im + smem_cap);
    const cta::Bufs g = desc_bufs(d, cur);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      A.lo[i] = g.lo[i];
      A.hi[i] = KW == 2 ? g.hi[i] : 0ull;
      A.re[i] = g.re[i];
      A.im[i] = g.im[i];
    }
    __syncthreads();
    done = cta::run_passes<KW>(d.plan, passes, p0, p1, A, B, n, d.capacity, stab, 4 * smem_cap,
                               warp_sums, &upd);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      g.lo[i] = A.lo[i];
      g.hi[i] = A.hi[i];   // zero for 64-bit labels: the buffers always hold valid high words
      g.re[i] = A.re[i];
      g.im[i] = A.im[i];
    }
  } else {
    cta::Bufs A = desc_bufs(d, cur), B = desc_bufs(d, cur ^ 1u);
    done = cta::run_passes<KW>(d.plan, passes, p0, p1, A, B, n, d.capacity, gtab, gtab_slots,
                               warp_sums, &upd);
    cur = A.lo == d.lo[1] ? 1u : 0u;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    dp->nnz = n;
    dp->cur = cur;
    dp->next_pass = p0 + done;
    // a failing branching pass was counted before it failed: take it back
    dp->updates += p0 + done < p1 ? upd - (uint64_t)n : upd;
    if (p0 + done < p1) {
      dp->status = SPS_ERR_CAPACITY;
      dp->failed_pass = p0 + done;
    }
    __threadfence();
  }
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT) k_batch(BatchDesc* desc, const uint32_t* order,
                                                uint32_t ncirc, uint32_t* head, uint32_t* gtabs,
                                                uint32_t gtab_slots, uint32_t max_passes,
                                                uint32_t smem_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t warp_sums[33];
  __shared__ uint32_t s_next;
  uint32_t* gtab = gtabs + (size_t)blockIdx.x * gtab_slots;
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(head, 1u);
    __syncthreads();
    const uint32_t c = s_next;
    __syncthreads();
    if (c >= ncirc) break;
    BatchDesc* dp = desc + order[c];
    if (dp->status != 0u || dp->next_pass >= dp->npasses) continue;
    if (dp->kw == 1)
      run_circuit<1>(dp, max_passes, smem_cap, smem, gtab, gtab_slots, warp_sums);
    else
      run_circuit<2>(dp, max_passes, smem_cap, smem, gtab, gtab_slots, warp_sums);
    __syncthreads();
  }
}

__global__ void k_batch_reset(BatchDesc* desc, uint32_t ncirc) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncirc) return;
  BatchDesc* d = desc + i;
  d->lo[0][0] = 0ull;
  d->hi[0][0] = 0ull;
  d->re[0][0] = 1.0;
  d->im[0][0] = 0.0;
  d->nnz = 1ull;
  d->cur = 0u;
  d->next_pass = 0u;
  d->status = 0u;
  d->failed_pass = 0u;
  d->updates = 0ull;
}

}  // namespace

int launch_batch_reset(void* stream, BatchDesc* desc, uint32_t ncirc) {
  if (ncirc == 0) return 0;
  k_batch_reset<<<(ncirc + 255) / 256, 256, 0, (cudaStream_t)stream>>>(desc, ncirc);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

size_t batch_smem_bytes(uint32_t smem_cap) { return (size_t)smem_cap * (64 + 16); }

int batch_kernel_attr(const BatchConfig& cfg) {
  const int smem = (int)batch_smem_bytes(cfg.smem_cap);
  const cudaError_t e =
      cfg.threads <= 256   ? cudaFuncSetAttribute(k_batch<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
      : cfg.threads <= 512 ? cudaFuncSetAttribute(k_batch<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                           : cudaFuncSetAttribute(k_batch<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e == cudaSuccess ? 0 : -1;
}

int launch_batch(void* stream, int sms, const BatchConfig& cfg, BatchDesc* desc,
                 const uint32_t* order, uint32_t ncirc, uint32_t* head, uint32_t* gtabs,
                 uint32_t gtab_slots, uint32_t max_passes, bool set_attr) {
  const size_t smem = batch_smem_bytes(cfg.smem_cap);
  const int blocks = sms * (int)cfg.blocks_per_sm;
  cudaStream_t st = (cudaStream_t)stream;
  if (set_attr && batch_kernel_attr(cfg) < 0) return -1;
  if (cfg.threads <= 256)
    k_batch<256><<<blocks, cfg.threads, smem, st>>>(desc, order, ncirc, head, gtabs, gtab_slots,
                                                    max_passes, cfg.smem_cap);
  else if (cfg.threads <= 512)
    k_batch<512><<<blocks, cfg.threads, smem, st>>>(desc, order, ncirc, head, gtabs, gtab_slots,
                                                    max_passes, cfg.smem_cap);
  else
    k_batch<1024><<<blocks, cfg.threads, smem, st>>>(desc, order, ncirc, head, gtabs, gtab_slots,
                                                     max_passes, cfg.smem_cap);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

bool batch_config_ok(const BatchConfig& c) {
  if (c.threads != 256 && c.threads != 512 && c.threads != 1024) return false;
  if (c.blocks_per_sm < 1 || c.blocks_per_sm > 4) return false;
  if (c.smem_cap != 0 && (c.smem_cap < 64 || c.smem_cap > 2048 || (c.smem_cap & (c.smem_cap - 1))))
    return false;
  if (batch_smem_bytes(c.smem_cap) * c.blocks_per_sm > 220 * 1024) return false;
  return true;
}

// ---- host side of a compiled circuit -----------------------------------------------
void pack_circuit(const std::vector<Pass>& passes, double eps, std::vector<unsigned char>* blob,
                  uint32_t* pass_off, uint64_t* work, uint64_t capacity) {
  auto put = [&](const void* src, size_t bytes) {
    const size_t at = blob->size();
    blob->resize((at + bytes + 15) & ~(size_t)15, 0);
    std::memcpy(blob->data() + at, src, bytes);
    return at;
  };
  std::vector<RunPass> recs(passes.size());
  uint64_t bound = 1, w = 0;
  for (size_t k = 0; k < passes.size(); ++k) {
    const Pass& p = passes[k];
    RunPass& r = recs[k];
    std::memset(&r, 0, sizeof(r));
    r.kind = p.kind;
    r.pass_serial = (uint32_t)k;
    r.fail_tag = p.first_gate;
    r.eps2 = eps * eps;
    r.eps = eps;
    if (p.kind == PASS_FUSED) {
      r.nops = p.ngates;
      r.flags = (p.has_perm ? 1u : 0u) | (p.has_phase ? 2u : 0u);
      r.nwords = (uint32_t)p.words.size();
      r.ops_off = (uint32_t)put(p.words.data(), p.words.size() * sizeof(OpWord));
      r.ph_off = p.ftab.empty() ? 0u
                                : (uint32_t)put(p.ftab.data(), p.ftab.size() * sizeof(double));
      w += bound * (uint64_t)p.ops.size();
    } else {
      r.br_off = (uint32_t)put(&p.br, sizeof(BranchOp));
      bound = std::min<uint64_t>(2 * bound, capacity);
      w += bound * 8;
    }
  }
  *pass_off = (uint32_t)put(recs.data(), recs.size() * sizeof(RunPass));
  *work = w;
}

}  // namespace sps

// ---- C ABI -------------------------------------------------------------------------
using namespace sps;

struct sps_batch {
  cudaStream_t stream = nullptr;
  int device = 0, sms = 0;
  BatchConfig cfg{512, 2, 1024, 0};
  struct Circ {
    uint32_t nqubits;
    uint64_t capacity;
    double eps;
    std::vector<Pass> passes;
    uint64_t work = 0;
    uint32_t pass_off = 0;
    std::vector<size_t> first_gate;
  };
  std::vector<Circ> circs;
  bool built = false;
  // device
  unsigned char* plan = nullptr;
  unsigned char* states = nullptr;
  BatchDesc* desc = nullptr;
  uint32_t* order = nullptr;
  uint32_t* head = nullptr;
  uint32_t* gtabs = nullptr;
  uint32_t gtab_slots = 0;
  size_t gtab_blocks = 0;
  struct Alloc {
    void* p;
    size_t bytes;
  };
  std::vector<Alloc> allocs;
  std::vector<BatchDesc> host_desc;   // descriptors as uploaded
  std::vector<BatchDesc> result;      // after sync
  uint64_t launches = 0;
  // one step (reset + persistent launch) captured as a CUDA graph
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  uint32_t g_passes = 0;
  BatchConfig g_cfg{0, 0, 0, 0};
};

namespace {

void drop_graph(sps_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  cudaGetLastError();
}

void batch_free(sps_batch* b) {
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (auto& a : b->allocs) hook_free(a.p, a.bytes, b->stream);
  b->allocs.clear();
  cudaStreamSynchronize(b->stream);
  b->plan = b->states = nullptr;
  b->desc = nullptr;
  b->order = b->head = b->gtabs = nullptr;
  cudaGetLastError();
}

sps_status cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return SPS_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? SPS_ERR_OOM : SPS_ERR_CUDA;
}

template <typename T>
sps_status balloc(sps_batch* b, T** out, size_t bytes) {
  void* p = hook_alloc(bytes, b->stream);
  if (!p) return SPS_ERR_OOM;
  b->allocs.push_back({p, bytes});
  *out = static_cast<T*>(p);
  return SPS_OK;
}

void bfree(sps_batch* b, void* p) {
  for (auto it = b->allocs.begin(); it != b->allocs.end(); ++it) {
    if (it->p == p) {
      hook_free(it->p, it->bytes, b->stream);
      b->allocs.erase(it);
      return;
    }
  }
}

// Per-block index tables for circuits whose state is kept in global memory.
sps_status ensure_gtabs(sps_batch* b) {
  uint64_t cap_max = 0;
  for (const auto& c : b->circs)
    if (c.capacity > b->cfg.smem_cap) cap_max = std::max(cap_max, c.capacity);
  uint32_t slots = 256;
  while (slots < 4 * cap_max) slots <<= 1;
  const size_t blocks = (size_t)b->sms * b->cfg.blocks_per_sm;
  if (b->gtabs && slots <= b->gtab_slots && blocks <= b->gtab_blocks) return SPS_OK;
  if (b->gtabs) bfree(b, b->gtabs);
  b->gtabs = nullptr;
  sps_status st = balloc(b, &b->gtabs, sizeof(uint32_t) * slots * blocks);
  if (st != SPS_OK) return st;
  b->gtab_slots = slots;
  b->gtab_blocks = blocks;
  return SPS_OK;
}

// Allocates and fills the plan, the state buffers and the descriptors.
sps_status batch_build(sps_batch* b) {
  if (b->built) return SPS_OK;
  std::vector<unsigned char> blob;
  for (auto& c : b->circs) pack_circuit(c.passes, c.eps, &blob, &c.pass_off, &c.work, c.capacity);
  size_t state_bytes = 0;
  std::vector<size_t> state_off(b->circs.size());
  for (size_t i = 0; i < b->circs.size(); ++i) {
    state_off[i] = state_bytes;
    state_bytes += 64 * (size_t)b->circs[i].capacity;   // two buffers of lo, hi, re, im
  }
  sps_status st;
  if ((st = balloc(b, &b->plan, std::max<size_t>(blob.size(), 16))) != SPS_OK) return st;
  if ((st = balloc(b, &b->states, std::max<size_t>(state_bytes, 64))) != SPS_OK) return st;
  if ((st = balloc(b, &b->desc, sizeof(BatchDesc) * std::max<size_t>(b->circs.size(), 1))) != SPS_OK)
    return st;
  if ((st = balloc(b, &b->order, sizeof(uint32_t) * std::max<size_t>(b->circs.size(), 1))) != SPS_OK)
    return st;
  if ((st = balloc(b, &b->head, 256)) != SPS_OK) return st;
  if ((st = ensure_gtabs(b)) != SPS_OK) return st;
  if (!blob.empty() &&
      (st = cuda_st(cudaMemcpyAsync(b->plan, blob.data(), blob.size(), cudaMemcpyHostToDevice,
                                    b->stream))) != SPS_OK)
    return st;
  b->host_desc.assign(b->circs.size(), BatchDesc());
  for (size_t i = 0; i < b->circs.size(); ++i) {
    const auto& c = b->circs[i];
    BatchDesc& d = b->host_desc[i];
    std::memset(&d, 0, sizeof(d));
    const size_t cap = c.capacity;
    unsigned char* base = b->states + state_off[i];
    for (int k = 0; k < 2; ++k) {
      unsigned char* bb = base + (size_t)k * 32 * cap;
      d.lo[k] = reinterpret_cast<uint64_t*>(bb);
      d.hi[k] = reinterpret_cast<uint64_t*>(bb + 8 * cap);
      d.re[k] = reinterpret_cast<double*>(bb + 16 * cap);
      d.im[k] = reinterpret_cast<double*>(bb + 24 * cap);
    }
    d.plan = b->plan;
    d.pass_off = c.pass_off;
    d.npasses = (uint32_t)c.passes.size();
    d.kw = c.nqubits <= 63 ? 1u : 2u;
    d.capacity = c.capacity;
  }
  // order: largest estimated work first
  std::vector<uint32_t> ord(b->circs.size());
  for (uint32_t i = 0; i < ord.size(); ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(),
                   [&](uint32_t x, uint32_t y) { return b->circs[x].work > b->circs[y].work; });
  if (!ord.empty() &&
      (st = cuda_st(cudaMemcpyAsync(b->order, ord.data(), sizeof(uint32_t) * ord.size(),
                                    cudaMemcpyHostToDevice, b->stream))) != SPS_OK)
    return st;
  if (!b->host_desc.empty() &&
      (st = cuda_st(cudaMemcpyAsync(b->desc, b->host_desc.data(),
                                    sizeof(BatchDesc) * b->host_desc.size(),
                                    cudaMemcpyHostToDevice, b->stream))) != SPS_OK)
    return st;
  if ((st = cuda_st(cudaStreamSynchronize(b->stream))) != SPS_OK) return st;
  b->built = true;
  return sps_batch_reset(b);
}

}  // namespace

extern "C" {

sps_status sps_batch_create(void* cuda_stream, sps_batch** out) {
  if (!out) return SPS_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return SPS_ERR_NO_DEVICE;
  }
  sps_batch* b = new (std::nothrow) sps_batch;
  if (!b) return SPS_ERR_OOM;
  b->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&b->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return SPS_ERR_CUDA;
  }
  *out = b;
  return SPS_OK;
}

void sps_batch_destroy(sps_batch* b) {
  if (!b) return;
  batch_free(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

sps_status sps_batch_add(sps_batch* b, uint32_t nqubits, uint64_t capacity, const sps_gate* gates,
                         size_t ngates, double prune_eps, uint32_t* index, size_t* failed_gate) {
  if (!b || b->built || nqubits < 1 || nqubits > 127 || capacity < 1 || capacity > (1u << 24) ||
      (ngates && !gates) || !(prune_eps >= 0.0))
    return SPS_ERR_ARG;
  sps_batch::Circ c;
  c.nqubits = nqubits;
  c.capacity = capacity;
  c.eps = prune_eps;
  size_t bad = 0;
  const sps_status st = compile(gates, ngates, nqubits, 0, &c.passes, &bad);
  if (st != SPS_OK) {
    if (failed_gate) *failed_gate = bad;
    return st;
  }
  if (index) *index = (uint32_t)b->circs.size();
  b->circs.push_back(std::move(c));
  return SPS_OK;
}

sps_status sps_batch_reset(sps_batch* b) {
  if (!b) return SPS_ERR_ARG;
  if (!b->built) return batch_build(b);
  if (launch_batch_reset(b->stream, b->desc, (uint32_t)b->circs.size()) < 0)
    return cuda_st(cudaGetLastError());
  return SPS_OK;
}

sps_status sps_batch_run(sps_batch* b, uint32_t max_passes) {
  if (!b) return SPS_ERR_ARG;
  if (!b->built) {
    const sps_status st = batch_build(b);
    if (st != SPS_OK) return st;
  }
  if (b->circs.empty()) return SPS_OK;
  if (cudaMemsetAsync(b->head, 0, sizeof(uint32_t), b->stream) != cudaSuccess)
    return cuda_st(cudaGetLastError());
  if (launch_batch(b->stream, b->sms, b->cfg, b->desc, b->order, (uint32_t)b->circs.size(), b->head,
                   b->gtabs, b->gtab_slots, max_passes) < 0)
    return cuda_st(cudaGetLastError());
  ++b->launches;
  return SPS_OK;
}

sps_status sps_batch_run_graph(sps_batch* b, uint32_t max_passes) {
  if (!b) return SPS_ERR_ARG;
  if (!b->built) {
    const sps_status st = batch_build(b);
    if (st != SPS_OK) return st;
  }
  if (b->circs.empty()) return SPS_OK;
  const BatchConfig& c = b->cfg;
  if (b->gexec && (max_passes != b->g_passes || c.threads != b->g_cfg.threads ||
                   c.blocks_per_sm != b->g_cfg.blocks_per_sm || c.smem_cap != b->g_cfg.smem_cap))
    drop_graph(b);
  if (!b->gexec) {
    if (!b->cap_stream &&
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return cuda_st(cudaGetLastError());
    if (batch_kernel_attr(c) < 0) return cuda_st(cudaGetLastError());
    const uint32_t n = (uint32_t)b->circs.size();
    if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return cuda_st(cudaGetLastError());
    bool ok = launch_batch_reset(b->cap_stream, b->desc, n) >= 0 &&
              cudaMemsetAsync(b->head, 0, sizeof(uint32_t), b->cap_stream) == cudaSuccess &&
              launch_batch(b->cap_stream, b->sms, c, b->desc, b->order, n, b->head, b->gtabs,
                           b->gtab_slots, max_passes, false) >= 0;
    cudaGraph_t g = nullptr;
    ok = cudaStreamEndCapture(b->cap_stream, &g) == cudaSuccess && ok;
    if (ok && cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) ok = false;
    b->graph = g;
    if (!ok) {
      drop_graph(b);
      return SPS_ERR_CUDA;
    }
    b->g_passes = max_passes;
    b->g_cfg = c;
  }
  if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess) return cuda_st(cudaGetLastError());
  ++b->launches;
  return SPS_OK;
}

sps_status sps_batch_sync(sps_batch* b, uint32_t* unfinished) {
  if (!b) return SPS_ERR_ARG;
  if (!b->built) return SPS_ERR_ARG;
  b->result.resize(b->circs.size());
  if (!b->result.empty() &&
      cudaMemcpyAsync(b->result.data(), b->desc, sizeof(BatchDesc) * b->result.size(),
                      cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
    return cuda_st(cudaGetLastError());
  const sps_status st = cuda_st(cudaStreamSynchronize(b->stream));
  if (st != SPS_OK) return st;
  if (unfinished) {
    uint32_t u = 0;
    for (const auto& d : b->result) u += (d.status == 0 && d.next_pass < d.npasses) ? 1u : 0u;
    *unfinished = u;
  }
  return SPS_OK;
}

sps_status sps_batch_circuit_status(sps_batch* b, uint32_t index, sps_status* status,
                                    size_t* failed_gate, uint64_t* nnz, int* finished) {
  if (!b || index >= b->circs.size() || index >= b->result.size()) return SPS_ERR_ARG;
  const BatchDesc& d = b->result[index];
  if (status) *status = (sps_status)d.status;
  if (failed_gate)
    *failed_gate = d.status && d.failed_pass < b->circs[index].passes.size()
                       ? b->circs[index].passes[d.failed_pass].first_gate
                       : 0;
  if (nnz) *nnz = d.nnz;
  if (finished) *finished = (d.status != 0 || d.next_pass >= d.npasses) ? 1 : 0;
  return SPS_OK;
}

sps_status sps_batch_get_amplitudes(sps_batch* b, uint32_t index, uint64_t* key_hi,
                                    uint64_t* key_lo, double* re, double* im, uint64_t cap,
                                    uint64_t* nnz_out) {
  if (!b || !key_lo || !re || !im || !nnz_out || index >= b->result.size()) return SPS_ERR_ARG;
  const BatchDesc& d = b->result[index];
  *nnz_out = d.nnz;
  if (d.nnz > cap) return SPS_ERR_CAPACITY;
  if (d.nnz == 0) return SPS_OK;
  const unsigned c = d.cur;
  const size_t bytes = 8 * d.nnz;
  bool ok = cudaMemcpyAsync(key_lo, d.lo[c], bytes, cudaMemcpyDefault, b->stream) == cudaSuccess &&
            cudaMemcpyAsync(re, d.re[c], bytes, cudaMemcpyDefault, b->stream) == cudaSuccess &&
            cudaMemcpyAsync(im, d.im[c], bytes, cudaMemcpyDefault, b->stream) == cudaSuccess;
  if (ok && key_hi) {
    if (d.kw == 2) {
      ok = cudaMemcpyAsync(key_hi, d.hi[c], bytes, cudaMemcpyDefault, b->stream) == cudaSuccess;
    } else {
      cudaPointerAttributes at;
      const bool dev = cudaPointerGetAttributes(&at, key_hi) == cudaSuccess &&
                       (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
      cudaGetLastError();
      if (dev)
        ok = cudaMemsetAsync(key_hi, 0, bytes, b->stream) == cudaSuccess;
      else
        std::memset(key_hi, 0, bytes);
    }
  }
  if (!ok) return cuda_st(cudaGetLastError());
  return cuda_st(cudaStreamSynchronize(b->stream));
}

sps_status sps_batch_set_config(sps_batch* b, const sps_batch_config* cfg) {
  if (!b || !cfg) return SPS_ERR_ARG;
  BatchConfig c{cfg->threads, cfg->blocks_per_sm, cfg->smem_cap, 0};
  if (!batch_config_ok(c)) return SPS_ERR_ARG;
  b->cfg = c;
  if (b->built) return ensure_gtabs(b);
  return SPS_OK;
}

sps_status sps_batch_get_config(sps_batch* b, sps_batch_config* cfg) {
  if (!b || !cfg) return SPS_ERR_ARG;
  cfg->threads = b->cfg.threads;
  cfg->blocks_per_sm = b->cfg.blocks_per_sm;
  cfg->smem_cap = b->cfg.smem_cap;
  cfg->reserved = 0;
  return SPS_OK;
}

sps_status sps_batch_tune(sps_batch* b, uint32_t repeats, sps_batch_config* best, float* best_ms) {
  if (!b) return SPS_ERR_ARG;
  if (!b->built) {
    const sps_status st = batch_build(b);
    if (st != SPS_OK) return st;
  }
  static const BatchConfig cands[] = {
      {256, 4, 256, 0},  {256, 2, 1024, 0}, {512, 2, 512, 0},   {512, 2, 1024, 0},
      {512, 1, 2048, 0}, {1024, 1, 1024, 0}, {1024, 1, 2048, 0}, {1024, 2, 1024, 0}};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_st(cudaGetLastError());
  float best_t = 1e30f;
  BatchConfig keep = b->cfg, win = b->cfg;
  if (repeats < 1) repeats = 1;
  for (const BatchConfig& c : cands) {
    if (!batch_config_ok(c)) continue;
    b->cfg = c;
    sps_status st = ensure_gtabs(b);
    if (st != SPS_OK) break;
    float tsum = 0.0f;
    bool skip = false;
    for (uint32_t r = 0; r < repeats; ++r) {
      if ((st = sps_batch_reset(b)) != SPS_OK) break;
      cudaEventRecord(e0, b->stream);
      if ((st = sps_batch_run(b, 0)) != SPS_OK) {
        // a configuration this device cannot launch is skipped, not fatal
        if (st == SPS_ERR_CUDA && cudaStreamSynchronize(b->stream) == cudaSuccess) {
          st = SPS_OK;
          skip = true;
        }
        break;
      }
      cudaEventRecord(e1, b->stream);
      if ((st = cuda_st(cudaEventSynchronize(e1))) != SPS_OK) break;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      tsum += ms;
    }
    if (st != SPS_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      b->cfg = keep;
      return st;
    }
    if (skip) continue;
    if (tsum / repeats < best_t) {
      best_t = tsum / repeats;
      win = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cfg = win;
  sps_status st = ensure_gtabs(b);
  if (st == SPS_OK) st = sps_batch_reset(b);
  if (best) {
    best->threads = win.threads;
    best->blocks_per_sm = win.blocks_per_sm;
    best->smem_cap = win.smem_cap;
    best->reserved = 0;
  }
  if (best_ms) *best_ms = best_t;
  return st;
}

sps_status sps_batch_counts(sps_batch* b, uint32_t* ncircuits, uint64_t* launches) {
  if (!b) return SPS_ERR_ARG;
  if (ncircuits) *ncircuits = (uint32_t)b->circs.size();
  if (launches) *launches = b->launches;
  return SPS_OK;
}

sps_status sps_batch_updates(sps_batch* b, uint64_t* total) {
  if (!b || !total) return SPS_ERR_ARG;
  uint64_t t = 0;
  for (const auto& d : b->result) t += d.updates;
  *total = t;
  return SPS_OK;
}

}  // extern "C"
