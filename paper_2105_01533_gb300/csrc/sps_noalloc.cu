// sps_branch_apply_static: one branching gate on caller-owned device arrays,
// with the hash table and control block in a fixed, file-scope device array
// instead of memory allocated at run time.
//
// Who needs it: callers that may not allocate device memory themselves or
// through a library - for example a host framework that owns every byte of
// device memory and forbids libraries from calling cudaMalloc, a service whose
// device footprint must be fixed when it starts, or code running inside an
// allocator callback, where allocating again would re-enter the allocator.
//
// The array below is part of the library image: every GPU that loads
// libsps.so holds it (8 MiB of table slots plus the 3,168-byte control block,
// 8,391,776 bytes in all) until the process exits.
#include <cuda_runtime.h>

#include <vector>

#include "sps.h"
#include "sps_internal.h"

namespace sps {
namespace {

constexpr uint32_t kStaticTableLog2 = 18;                 // 262,144 slots of 32 B = 8 MiB
constexpr uint64_t kStaticMaxInput = 1ull << 16;         // table holds 2 * n_in labels at <= 50% load

struct StaticScratch {
  Slot table[1u << kStaticTableLog2];
  Ctl ctl;
};
// the footprint the header states: keep the two in step
static_assert(sizeof(Ctl) == 3168, "control block size changed: update sps.h");
static_assert(sizeof(StaticScratch) == 8391776, "scratch size changed: update sps.h");

static __device__ __align__(256) StaticScratch g_static_scratch;

// Device address of the scratch array on the current device. Host code cannot
// use the symbol itself as a device address; the lookup is a host-side query
// (no stream operation) and is made on every call, so the address stays right
// if the device's context was reset and the module loaded again elsewhere.
sps_status static_scratch(int device, StaticScratch** out, int* sms) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return SPS_ERR_CUDA;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return SPS_ERR_CUDA;
  }
  *out = static_cast<StaticScratch*>(p);
  *sms = n;
  return SPS_OK;
}

}  // namespace
}  // namespace sps

using namespace sps;

extern "C" sps_status sps_branch_apply_static(
    const sps_gate* gate, uint32_t nqubits, const uint64_t* in_hi, const uint64_t* in_lo,
    const double* in_re, const double* in_im, uint64_t n_in, double prune_eps, uint64_t* out_hi,
    uint64_t* out_lo, double* out_re, double* out_im, uint64_t out_cap, uint64_t* n_out,
    void* cuda_stream) {
  if (!gate || !n_out || nqubits < 1 || nqubits > 127 || !(prune_eps >= 0.0)) return SPS_ERR_ARG;
  *n_out = 0;
  const int kw = nqubits <= 63 ? 1 : 2;
  if (n_in > kStaticMaxInput) return SPS_ERR_CAPACITY;
  if (n_in && (!in_lo || !in_re || !in_im || (kw == 2 && !in_hi))) return SPS_ERR_ARG;
  if (!out_lo || !out_re || !out_im || (kw == 2 && !out_hi)) return SPS_ERR_ARG;
  // outputs must not alias inputs: the compaction writes while the table
  // still refers to entries of the input arrays
  if (out_lo == in_lo || out_re == in_re || out_im == in_im || (kw == 2 && out_hi == in_hi))
    return SPS_ERR_ARG;
  // the gate must be a single valid two-nonzero gate
  std::vector<Pass> passes;
  size_t bad = 0;
  if (compile(gate, 1, nqubits, 0, &passes, &bad) != SPS_OK || passes.size() != 1 ||
      passes[0].kind != PASS_BRANCH)
    return SPS_ERR_ARG;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return SPS_ERR_NO_DEVICE;
  }
  StaticScratch* scratch = nullptr;
  int sms = 0;
  sps_status st = static_scratch(device, &scratch, &sms);
  if (st != SPS_OK) return st;

  Bufs bufs{};
  bufs.b[0].lo = const_cast<uint64_t*>(in_lo);
  bufs.b[0].hi = const_cast<uint64_t*>(in_hi);
  bufs.b[0].re = const_cast<double*>(in_re);
  bufs.b[0].im = const_cast<double*>(in_im);
  bufs.b[1].lo = out_lo;
  bufs.b[1].hi = out_hi;
  bufs.b[1].re = out_re;
  bufs.b[1].im = out_im;
  Ctl* ctl = &scratch->ctl;
  Slot* table = scratch->table;

  LaunchCfg lc;
  lc.threads = 256;
  lc.max_blocks = sms * 8;
  lc.stream = cuda_stream;

  BranchLaunch b;
  b.op = passes[0].br;
  b.eps = prune_eps;
  b.load_pct = 50;
  b.max_log2 = kStaticTableLog2;
  b.probe_limit = 1u << kStaticTableLog2;
  b.pass_serial = 1;
  b.coop = 1;
  b.capacity = out_cap;
  b.fail_tag = 0;
  MaskRing ring;
  const uint32_t mg_set = ring.writer();
  b.mg = ring.writer();

  // The array keeps the previous call's contents: reset the control block and
  // clear the part of the table this call uses before emitting into it.
  const uint64_t slots = 1ull << table_log2_for(n_in, b.load_pct, kStaticTableLog2);
  if (launch_table_clear(lc, table, slots) < 0 || launch_set_nnz(cuda_stream, ctl, n_in, mg_set) < 0 ||
      launch_branch_emit(lc, kw, ctl, bufs, table, b, n_in, nullptr) < 0 ||
      launch_branch_compact(lc, kw, ctl, bufs, table, b, n_in, nullptr) < 0) {
    cudaGetLastError();
    return SPS_ERR_CUDA;
  }
  Ctl result;
  if (cudaMemcpyAsync(&result, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                      (cudaStream_t)cuda_stream) != cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) {
    cudaGetLastError();
    return SPS_ERR_CUDA;
  }
  if (result.status != 0u) return (sps_status)result.status;
  *n_out = result.nnz;
  return SPS_OK;
}
