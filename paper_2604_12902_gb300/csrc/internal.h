// internal.h -- host-side declarations shared by the C-ABI layer and the
// kernel launchers (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "engine.cuh"

struct rasp_batch;
struct rasp_config;

namespace rasp {

struct StepVariant {
  bool masked;   // w < 64
  bool checked;  // RASP_CHECKED semantics
  bool hist;     // collect per-opcode counters
  bool vote;     // warp opcode voting instead of guarded selects
  bool classic;  // classic opcode set (Sec. 1.1: SUB, BPA); plain and HBM-slab persistent, select only
  bool block;    // HBM-slab persistent: one predicated block per step instead of the epoch loop;
                 // shared-program schedule: one step at a time per lane instead of the epoch loop
  bool narrow;   // M in 4-byte words (w <= 32): plain and HBM-slab persistent schedules
};

// Persistent-kernel launch shape for one bucket of VMs.
struct PersistShape {
  bool staged;          // M, tape and y in shared memory (bulk-copied)
  uint32_t ncap;        // slot capacity for M (words, even)
  uint32_t slot_words;  // words per lane slot (M + tape + y, padded)
  uint32_t warps;       // warps per CTA
  uint32_t epoch;       // steps between warp scheduling points
  uint32_t refill_min;  // idle lanes that trigger a refill (staged schedule)
  uint32_t idle_exit;   // HBM-slab epoch loop: stopped lanes that end an epoch early (0: never)
  bool block;           // one step at a time (the per-step form) instead of the epoch loop
  uint32_t grid;        // CTAs
  uint32_t ctas_per_sm; // resident CTAs per SM (occupancy)
  size_t smem;          // dynamic shared memory per CTA
};

// c_0 of every VM; with `lazy` the program words M[0, plen) are left
// unwritten (shared-program schedule: the steps read them from the program).
// The program words are read from prog32 (4-byte words, sign-extended) when
// it is not NULL, else from prog.
cudaError_t launch_pack(const DevState& S, const uint64_t* prog, const int32_t* prog32, const uint64_t* prog_off,
                        const uint32_t* prog_of_vm, uint32_t num_vms, uint64_t wmask, uint32_t sp,
                        bool lazy, cudaStream_t stream);

// Shared-program schedule: one CTA per program (program in shared memory),
// lanes run the program's VMs pv_ids[pv_off[p] .. pv_off[p+1]) (epoch loop
// for WRAP without counters, else one step at a time). The slabs of VMs
// with codedirty = 0 need not hold their program words.
cudaError_t launch_shared(const StepVariant& var, const DevState& S, const Params& P, const uint64_t* prog,
                          const uint64_t* prog_off, const uint32_t* pv_off, const uint32_t* pv_ids,
                          uint32_t num_programs, uint32_t max_plen, uint32_t epoch, cudaStream_t stream);

// M[0, plen) = the VM's program for every VM with codedirty = 0 (after a
// lazy pack, before anything but the shared-program kernel reads the slabs).
cudaError_t launch_materialize(const DevState& S, const uint64_t* prog, const uint64_t* prog_off,
                               const uint32_t* prog_of_vm, uint32_t num_vms, uint64_t wmask, cudaStream_t stream);

// One-time function attributes of the plain kernel (carveout).
void plain_configure(const StepVariant& var);

cudaError_t launch_plain(const StepVariant& var, const DevState& S, const Params& P,
                         const uint32_t* ids, uint32_t count, cudaStream_t stream);

// Fills grid/smem of `shape` for the current device (occupancy-sized) and
// returns the resident CTAs per SM (0 if the shape cannot launch).
int persist_configure(const StepVariant& var, PersistShape& shape);

cudaError_t launch_persist(const StepVariant& var, const DevState& S, const Params& P, const Queue& Q,
                           const PersistShape& shape, cudaStream_t stream);

// Halting-time histogram (device): counts[nbins] of HALTED VMs by
// edges[k] <= steps < edges[k+1]; other[4] = RUNNING, TIMEOUT, faulted,
// HALTED outside the edges. edges, counts, other are device pointers.
constexpr uint32_t kMaxHistBins = 4096;
cudaError_t launch_tau_hist(const DevState& S, uint32_t num_vms, const uint64_t* edges, uint32_t nbins,
                            unsigned long long* counts, unsigned long long* other, cudaStream_t stream);

// Dense list of the still-RUNNING VMs among ids[0, count): out[0, *out_count).
cudaError_t launch_compact(const uint32_t* ids, uint32_t count, const uint8_t* status, uint32_t* out,
                           uint32_t* out_count, cudaStream_t stream);

// Top-k halting times: candidate (tau_h, VM id); ok = 0 marks an empty slot.
struct TopCand {
  uint64_t steps;
  uint32_t vm;
  uint32_t ok;
};
constexpr uint32_t kMaxTopK = 1024;
constexpr uint32_t kMaxTopBlocks = 256;
// best[0, k): the k HALTED VMs with the largest steps (ties: smaller id),
// best first, empty slots last; cand holds kMaxTopBlocks * k entries.
cudaError_t launch_topk(const DevState& S, uint32_t num_vms, uint32_t k, TopCand* cand, TopCand* best,
                        cudaStream_t stream);

// memset of device memory by a kernel of this library (falls back to
// cudaMemsetAsync for a pointer that is not 16-byte aligned).
cudaError_t fill_bytes(void* p, uint8_t value, uint64_t bytes, cudaStream_t stream);

// Host-side fault injection for tests: true when the environment variable
// RASP_FAULT_INJECT is "alloc", in which case every device allocation the
// library would make (a batch, the autotuner's snapshot, a pool arena)
// fails as if cudaMalloc had, with RASP_ENOMEM. Nothing reaches the GPU.
bool inject_alloc_failure();

// Host-side test hook: with RASP_FAULT_INJECT=wait the SMEM-staged kernel is
// launched with a bounded-wait limit of 0 polls, so its wait for each bulk
// copy gives up at once: the kernel flags ERR_WAIT_TIMEOUT (rasp_sync and
// rasp_read_state return RASP_EDEVICE), lets the copies it issued land
// (a wait with the default limit) and returns. No fault, no trap, no hang.
bool inject_wait_expiry();

// ---- serving: one persistent kernel over a ring of VMs shared by requests
// Device descriptor of one admitted request (a "slot"): its batch's state
// store, the budget of its run and the word written to its completion flag.
struct ServeSlot {
  DevState S;
  uint64_t budget;       // max_steps of the request's run
  uint32_t num_vms;      // entries with this slot index name VMs below this
  uint32_t gen;          // written to done[slot] when its last VM stops (nonzero)
};

struct ServeArgs {
  const ServeSlot* slots;
  uint32_t num_slots;
  uint32_t* pending;                 // [num_slots] VMs of the request not yet stopped
  const uint64_t* ring;              // entries (slot << 32 | vm), position p at ring[p & ring_mask]
  uint64_t ring_mask;
  unsigned long long* head;          // positions claimed by the kernel
  unsigned long long* credits;       // published entries not yet claimed (signed; may dip while a shortfall is returned)
  unsigned long long* state;         // warps holding work, | 1 << 63 once the instance closes (0 at launch)
  uint32_t* done;                    // host-mapped [num_slots] completion words
  const volatile uint32_t* launched; // host-mapped: instances the host has launched
  uint32_t* exited;                  // host-mapped: instances that have returned
  uint32_t instance;                 // this launch's number (1, 2, ...)
  uint32_t epoch;
  uint32_t idle_polls;               // empty-ring polls (1 to 16 us apart) before the newest instance returns
  int* err;                          // ERR_RING: a ring entry outside the slot table
};

// Serving kernel shape for the device: grid (leaving one CTA slot per SM
// free for the requests' pack and ring-fill kernels) and threads per CTA.
struct ServeShape {
  uint32_t grid;
  uint32_t threads;
};
int serve_configure(const StepVariant& var, ServeShape& sh);
cudaError_t launch_serve(const StepVariant& var, const ServeArgs& A, const Params& P, const ServeShape& sh,
                         cudaStream_t stream);
// ring[(start + k) & mask] = slot << 32 | ids[k] for k < count, then *credits += count
// (two launches on `stream`, so every entry is written before it can be claimed).
cudaError_t launch_ring_append(uint64_t* ring, uint64_t mask, unsigned long long start, uint32_t slot,
                               const uint32_t* ids, uint32_t count, unsigned long long* credits,
                               cudaStream_t stream);

// rasp_load_programs from 8-byte (word_size 8) or 4-byte (word_size 4) words.
int load_programs(rasp_batch* b, const void* words, int word_size, const uint64_t* offsets, uint64_t num_programs,
                  const uint32_t* prog_of_vm);

// dst[k] = src[k] sign-extended, k < count (device pointers, 16-byte aligned).
cudaError_t launch_widen(const int32_t* src, uint64_t* dst, uint64_t count, cudaStream_t stream);

// rasp_batch_create; with plan = false the launch plan is left to the first
// rasp_run (the serving pool's batches are never run by rasp_run).
int create_batch(const rasp_config* cfg, uint64_t num_vms, const uint32_t* mem_words, bool plan,
                 rasp_batch** out);

// The state store and step parameters of a batch (for the serving pool).
const DevState& batch_dev_state(const rasp_batch* b);
Params batch_params(const rasp_batch* b);
const uint32_t* batch_queue(const rasp_batch* b);   // VM ids in the batch's queue order (device)

// Aggregate: out[0] = sum steps, out[1..5] = count per status.
cudaError_t launch_stats(const DevState& S, uint32_t num_vms, unsigned long long* out, cudaStream_t stream);

}  // namespace rasp
