// static_run.cu -- rasp_run_static: run a caller-owned state store without
// allocating anything.
//
// Some callers cannot call cudaMalloc (or any allocator) at the moment they
// want to run machines: engines whose device memory is owned and accounted
// by another framework's allocator (a cudaMalloc behind its back breaks its
// accounting and can fail when that allocator holds the free memory), and
// real-time loops where an allocation, and the device-wide synchronisation
// cudaMalloc/cudaFree can cause, is not allowed. rasp_run_static serves
// them: the caller passes device pointers to its own state store and the
// call allocates no device or host memory.
//
// The only memory it needs beyond the caller's buffers is a work queue of
// VM ids plus a few counters. That scratch is the file-scope array
// g_static_scratch below, a fixed RASP_STATIC_MAX_VMS entries big, which
// every GPU that loads the library keeps until the process exits. In host
// code the array's name is only a host-side stand-in, so the first call on
// each device looks up its device address with cudaGetSymbolAddress (with
// that device current) and passes that address to the kernels.
//
// The caller's per-VM layout (n, mem_off) lives in device memory, where the
// host cannot check it without a copy. The queueing kernel checks it per VM
// instead: a VM whose n is outside 1..2^31-1, whose mem_off is odd, or whose
// slab does not lie inside mem[0, mem_words) is not queued (so no kernel
// ever reads or writes outside the caller's buffers for it) and is counted
// in the caller's optional `rejected` word.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/rasp.h"
#include "engine.cuh"

namespace rasp {
namespace {

constexpr uint32_t kHeader = 64;   // words before the id queue: [0] queued VMs, [1] queue head
constexpr uint32_t kMaxDevices = 64;

static __device__ __align__(256) uint32_t g_static_scratch[kHeader + RASP_STATIC_MAX_VMS];

struct DeviceSetup {
  bool done = false;
  uint32_t* scratch = nullptr;   // device address of g_static_scratch on this device
  int sms = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

int report(const rasp_static_run* r, int code, const char* fmt, ...) {
  if (r && r->err_buf && r->err_buf_size) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(r->err_buf, r->err_buf_size, fmt, ap);   // fixed caller buffer: no allocation
    va_end(ap);
  }
  return code;
}

// Queue the ids of the machines that are still RUNNING and whose memory
// layout is valid (warp-aggregated); count the RUNNING machines refused for
// their layout in *rejected (if given).
__global__ void __launch_bounds__(256) k_static_compact(const uint8_t* __restrict__ status,
                                                        const uint32_t* __restrict__ n,
                                                        const uint64_t* __restrict__ mem_off, uint32_t num_vms,
                                                        uint64_t mem_words, uint32_t* __restrict__ scratch,
                                                        uint32_t* __restrict__ rejected) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < num_vms; base += stride) {
    const uint32_t v = base + threadIdx.x;
    bool run = v < num_vms && status[v] == ST_RUNNING;
    bool bad = false;
    if (run) {
      // the slab is read in aligned 16-byte pairs, so its even-padded length
      // must fit: mem_off even, 1 <= n < 2^31, mem_off + even(n) <= mem_words
      const uint64_t nn = n[v], off = mem_off[v];
      const uint64_t npad = (nn + 1ull) & ~1ull;
      bad = nn == 0ull || nn >= (1ull << 31) || (off & 1ull) || off > mem_words || npad > mem_words - off;
      run = !bad;
    }
    const uint32_t m = __ballot_sync(0xffffffffu, run);
    const uint32_t mb = __ballot_sync(0xffffffffu, bad);
    uint32_t first = 0;
    if (lane == 0 && m) first = atomicAdd(&scratch[0], (uint32_t)__popc(m));
    if (lane == 0 && mb && rejected) atomicAdd(rejected, (uint32_t)__popc(mb));
    first = __shfl_sync(0xffffffffu, first, 0);
    if (run) scratch[kHeader + first + __popc(m & ((1u << lane) - 1u))] = v;
  }
}

// Persistent warps over the queued ids: each lane runs one VM (memory in
// HBM) until it stops, then the warp claims new ids for its idle lanes.
template <bool MASKED, bool CHECKED>
__global__ void __launch_bounds__(128) k_static_persist(DevState S, Params P, uint32_t* __restrict__ scratch,
                                                        uint32_t epoch) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t count = *reinterpret_cast<volatile uint32_t*>(&scratch[0]);
  Hist h;
  h.zero();
  Regs r{};
  r.n = 1;
  int32_t vm = -1;
  bool active = false, exhausted = false;
  uint32_t final_st = ST_RUNNING;
  uint64_t* M = S.mem;
  const uint64_t* T = S.tape;
  uint64_t* Y = S.y;
  for (;;) {
    const bool need = (vm < 0) && !exhausted;
    const uint32_t needm = __ballot_sync(0xffffffffu, need);
    if (needm) {
      const int leader = __ffs(needm) - 1;
      uint32_t base = 0;
      if ((int)lane == leader) base = atomicAdd(&scratch[1], (uint32_t)__popc(needm));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const uint32_t pos = base + (uint32_t)__popc(needm & ((1u << lane) - 1u));
        if (pos < count) {
          vm = (int32_t)scratch[kHeader + pos];
          load_regs(S, P, (uint32_t)vm, r);
          arm_regs(P, r);
          M = S.mem + S.mem_off[vm];
          T = S.tape + (uint64_t)vm * P.ellp;
          Y = S.y + (uint64_t)vm * P.sp;
          active = true;
        } else {
          exhausted = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, exhausted && !active)) break;
    if (active) {
      for (uint32_t t = 0; t < epoch; ++t) {
        const uint32_t s = one_step<MASKED, CHECKED, false, false>(M, T, Y, P, r, h);
        if (s != CONT) {
          active = false;
          final_st = s;
          break;
        }
      }
    }
    if (vm >= 0 && !active) {
      store_regs(S, (uint32_t)vm, r, final_st);
      vm = -1;
    }
  }
}

using StaticFn = void (*)(DevState, Params, uint32_t*, uint32_t);

StaticFn pick(bool masked, bool checked) {
  if (checked) return k_static_persist<false, true>;
  return masked ? k_static_persist<true, false> : k_static_persist<false, false>;
}

}  // namespace
}  // namespace rasp

using namespace rasp;

extern "C" int rasp_run_static(const rasp_static_run* r) {
  if (!r) return RASP_EINVAL;
  if (r->num_vms > RASP_STATIC_MAX_VMS)
    return report(r, RASP_EINVAL, "num_vms = %llu exceeds the static scratch capacity of %u VMs",
                  (unsigned long long)r->num_vms, (unsigned)RASP_STATIC_MAX_VMS);
  if (r->word_bits < 2 || r->word_bits > 64) return report(r, RASP_EINVAL, "word_bits must be in 2..64");
  if (r->semantics != RASP_WRAP && r->semantics != RASP_CHECKED) return report(r, RASP_EINVAL, "unknown semantics");
  if (r->semantics == RASP_CHECKED && r->word_bits != 64)
    return report(r, RASP_EINVAL, "CHECKED semantics needs word_bits = 64");
  if (r->num_vms == 0) return RASP_OK;
  if (!r->i || !r->a || !r->steps || !r->cap || !r->status || !r->uhead || !r->ylen || !r->n || !r->mem_off ||
      !r->mem || (r->in_cap && !r->tape) || (r->out_cap && !r->y))
    return report(r, RASP_EINVAL, "a state-store pointer is NULL");
  if (r->mem_words == 0) return report(r, RASP_EINVAL, "mem_words (the size of mem) must be given");
  if (reinterpret_cast<uintptr_t>(r->rejected) & 3u) return report(r, RASP_EINVAL, "rejected must be 4-byte aligned");
  if ((reinterpret_cast<uintptr_t>(r->mem) & 15u) || (reinterpret_cast<uintptr_t>(r->tape) & 15u) ||
      (reinterpret_cast<uintptr_t>(r->y) & 15u))
    return report(r, RASP_EINVAL, "mem, tape and y must be 16-byte aligned");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report(r, RASP_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= (int)kMaxDevices) return report(r, RASP_EINVAL, "device ordinal %d not supported", dev);
  const bool masked = r->word_bits < 64;
  const bool checked = r->semantics == RASP_CHECKED;
  const StaticFn fn = pick(masked, checked);
  DeviceSetup setup;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.done) {
      // once per device, with that device current: the device address of
      // the scratch array (its host-side name is not a device address)
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess) return report(r, RASP_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return report(r, RASP_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
      // load every kernel of this file now, so that no later call loads code
      cudaFuncAttributes fa;
      const void* fns[] = {(const void*)k_static_compact, (const void*)pick(false, false),
                           (const void*)pick(true, false), (const void*)pick(false, true)};
      for (const void* f : fns) {
        e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return report(r, RASP_ECUDA, "cudaFuncGetAttributes: %s", cudaGetErrorString(e));
      }
      s.scratch = static_cast<uint32_t*>(ptr);
      s.sms = sms;
      s.done = true;
    }
    setup = s;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 128, 0);
  if (e != cudaSuccess || per_sm <= 0) return report(r, RASP_ECUDA, "occupancy query failed");

  DevState S{};
  S.i = reinterpret_cast<uint64_t*>(r->i);
  S.a = reinterpret_cast<uint64_t*>(r->a);
  S.steps = r->steps;
  S.cap = r->cap;
  S.status = r->status;
  S.uhead = r->uhead;
  S.ylen = r->ylen;
  S.n = r->n;
  S.mem_off = r->mem_off;
  S.mem = reinterpret_cast<uint64_t*>(r->mem);
  S.tape = reinterpret_cast<const uint64_t*>(r->tape);
  S.y = reinterpret_cast<uint64_t*>(r->y);
  Params P{};
  P.wmask = masked ? ((1ull << r->word_bits) - 1ull) : ~0ull;
  P.budget = r->max_steps;
  P.ell = r->in_cap;
  P.s = r->out_cap;
  P.ellp = (r->in_cap + 1u) & ~1u;
  P.sp = (r->out_cap + 1u) & ~1u;
  P.err = nullptr;     // the static kernels have no bounded wait to report
  P.hist = nullptr;
  cudaStream_t stream = static_cast<cudaStream_t>(r->stream);

  // the queue counters start at zero on every call (the ids need no clearing)
  e = cudaMemsetAsync(setup.scratch, 0, kHeader * sizeof(uint32_t), stream);
  if (e == cudaSuccess && r->rejected) e = cudaMemsetAsync(r->rejected, 0, sizeof(uint32_t), stream);
  if (e != cudaSuccess) return report(r, RASP_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  const uint32_t V = (uint32_t)r->num_vms;
  uint32_t cblocks = (V + 255u) / 256u;
  if (cblocks > (uint32_t)setup.sms * 8u) cblocks = (uint32_t)setup.sms * 8u;
  k_static_compact<<<cblocks, 256, 0, stream>>>(r->status, r->n, r->mem_off, V, r->mem_words, setup.scratch,
                                                 r->rejected);
  uint32_t grid = (uint32_t)(per_sm * setup.sms);
  const uint32_t useful = (V + 127u) / 128u;
  if (grid > useful) grid = useful;
  fn<<<grid, 128, 0, stream>>>(S, P, setup.scratch, 64u);
  e = cudaGetLastError();
  if (e != cudaSuccess) return report(r, RASP_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
  return RASP_OK;
}
