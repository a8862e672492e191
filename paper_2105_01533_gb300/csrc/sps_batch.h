// Batched execution internals (shared by sps_batch.cu and the serving loop).
#pragma once

#include <cstdint>

#include "sps_internal.h"

namespace sps {

// One circuit of a batched launch. The kernel updates next_pass, nnz, cur,
// status and failed_pass in place.
struct BatchDesc {
  uint64_t* lo[2];
  uint64_t* hi[2];          // present for both label widths (zero high words)
  double* re[2];
  double* im[2];
  const unsigned char* plan;  // base of its RunPass records and payloads
  uint32_t pass_off;        // byte offset of the RunPass array within plan
  uint32_t npasses;
  uint32_t kw;              // label words: 1 or 2
  uint32_t next_pass;       // progress
  uint64_t capacity;
  uint64_t nnz;
  uint32_t cur;             // buffer holding the state
  uint32_t status;          // sps_status of the circuit (0 = fine)
  uint32_t failed_pass;
  uint32_t reserved;
  uint64_t updates;         // sum over applied gates of the nonzeros before the gate
};

struct BatchConfig {
  uint32_t threads;         // 256, 512 or 1024
  uint32_t blocks_per_sm;   // persistent blocks per SM
  uint32_t smem_cap;        // circuits with capacity <= this run in shared memory
  uint32_t reserved;
};

size_t batch_smem_bytes(uint32_t smem_cap);
bool batch_config_ok(const BatchConfig& c);
// set_attr: set the kernel's shared-memory attribute first (else the caller
// did, with batch_kernel_attr: not a stream operation, kept out of captures).
int launch_batch(void* stream, int sms, const BatchConfig& cfg, BatchDesc* desc,
                 const uint32_t* order, uint32_t ncirc, uint32_t* head, uint32_t* gtabs,
                 uint32_t gtab_slots, uint32_t max_passes, bool set_attr = true);
int batch_kernel_attr(const BatchConfig& cfg);
// Sets every listed circuit to |0...0> with no progress (one thread per circuit).
int launch_batch_reset(void* stream, BatchDesc* desc, uint32_t ncirc);
// Packs a compiled circuit's passes into blob; *pass_off locates its RunPass
// array, *work is its estimated work (entries x ops) for ordering.
void pack_circuit(const std::vector<Pass>& passes, double eps, std::vector<unsigned char>* blob,
                  uint32_t* pass_off, uint64_t* work, uint64_t capacity);

// Device memory through the library's allocator hook (sps_set_allocator).
void* hook_alloc(size_t bytes, void* stream);
void hook_free(void* p, size_t bytes, void* stream);

}  // namespace sps
