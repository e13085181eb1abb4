// kernels.cu -- sm_103a kernels of the batched word-RASP engine.
//
//   k_pack     c_0(P, x) for every VM (Sec. 2.1): M = P 0^(n-2m), y = 0,
//              i = a = steps = u_0 = y_0 = 0. One warp per VM, 16-byte stores.
//   k_plain    the plain form: one thread per VM, state in HBM, each VM run
//              until it stops, one launch per batch.
//   k_persist  persistent workers (cf. the striped workers of App. A,
//              Alg. 1) with a device-side queue: each lane runs one VM at a
//              time; lanes whose VM stopped are written back and refilled
//              from the queue at warp scheduling points. In the staged form
//              the lane's M, tape and outputs live in shared memory, moved
//              in and out by 1-D bulk async copies (cp.async.bulk).
//   k_stats    sum of steps and count per status.
//
// Steps are evaluated either in the guarded-sum (select) form of
// `one_step`, or, with the VOTE variant, by warp opcode voting: lanes are
// grouped by opcode with __match_any_sync and each group runs the handler of
// its case of the Sec. 2.1 equation.
#include <cstdio>

#include "engine.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace rasp {

constexpr uint32_t FULL = 0xffffffffu;
constexpr uint32_t WAIT_LIMIT = 1u << 22;   // mbarrier polls before giving up

// ------------------------------------------------------------------ pack
__global__ void __launch_bounds__(256) k_pack(DevState S, const uint64_t* __restrict__ prog,
                                              const uint64_t* __restrict__ prog_off,
                                              const uint32_t* __restrict__ prog_of_vm, uint32_t num_vms,
                                              uint64_t wmask, uint32_t sp) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < num_vms; v += warps) {
    const uint32_t p = prog_of_vm ? prog_of_vm[v] : v;
    const uint64_t po = prog_off[p];
    const uint64_t plen = prog_off[p + 1] - po;
    const uint64_t* src = prog + po;                   // po is even: 16-byte aligned
    uint64_t* dst = S.mem + S.mem_off[v];
    const uint32_t npad = (S.n[v] + 1u) & ~1u;
    for (uint32_t k = 2u * lane; k < npad; k += 64u) {
      ulonglong2 w;
      if (k + 1u < plen) {
        w = *reinterpret_cast<const ulonglong2*>(src + k);
        w.x &= wmask;
        w.y &= wmask;
      } else {
        w.x = (k < plen) ? (src[k] & wmask) : 0ull;
        w.y = 0ull;
      }
      *reinterpret_cast<ulonglong2*>(dst + k) = w;
    }
    uint64_t* Y = S.y + (uint64_t)v * sp;
    for (uint32_t k = lane; k < sp; k += 32u) Y[k] = 0ull;
    if (lane == 0) {
      S.i[v] = 0;
      S.a[v] = 0;
      S.steps[v] = 0;
      S.status[v] = ST_RUNNING;
      S.uhead[v] = 0;
      S.ylen[v] = 0;
    }
  }
}

// ------------------------------------------------------------------ vote step
// Warp-synchronous step: every lane of the warp calls it; `active` lanes
// take part. Returns CONT or a final status like one_step.
template <bool MASKED, bool CHECKED, bool HIST>
__device__ __forceinline__ uint32_t vote_step(uint64_t* __restrict__ M, const uint64_t* __restrict__ T,
                                              uint64_t* __restrict__ Y, const Params& P, Regs& r, Hist& h,
                                              bool active) {
  const uint64_t wm = MASKED ? P.wmask : ~0ull;
  const uint64_t i = r.i, a = r.a;
  const uint32_t ip = r.ip, n = r.n;
  uint32_t result = CONT;
  uint32_t op = 0;
  uint64_t j = 0;
  uint32_t jm = 0;
  if (active) {
    bool fetch_fault = false;
    if (CHECKED) fetch_fault = !(i < (uint64_t)n - 1);
    if (fetch_fault) {
      result = (r.steps >= r.stop) ? (r.steps >= r.cap ? ST_TIMEOUT : ST_RUNNING) : ST_FAULT_ADDR;
    } else {
      uint64_t o;
      if (!(ip & 1u) && ip + 1u < n && i != wm) {
        const ulonglong2 oj = *reinterpret_cast<const ulonglong2*>(M + ip);
        o = oj.x;
        j = oj.y;
      } else {
        o = M[ip];
        uint32_t k1 = (i == wm) ? 0u : ip + 1u;
        if (k1 == n) k1 = 0u;
        j = M[k1];
      }
      jm = mod_n(j, n);
      const bool valid = (o - 1ull) < 7ull;
      op = valid ? (uint32_t)o : 0u;
      const bool fixed = !valid || (op == 6u && r.u0 >= P.ell) || (op == 5u && a != 0 && j == i);
      if (fixed) result = ST_HALTED;
      else if (r.steps >= r.stop) result = r.steps >= r.cap ? ST_TIMEOUT : ST_RUNNING;
      else if (CHECKED && op != 1u && op != 5u && j >= (uint64_t)n) result = ST_FAULT_ADDR;
    }
  }
  const uint32_t exec_op = (active && result == CONT) ? op : 0u;
  uint32_t pend = __ballot_sync(FULL, exec_op != 0u);
  const uint32_t peers = __match_any_sync(FULL, exec_op);
  const uint32_t lane = threadIdx.x & 31u;
  bool taken = false;
  while (pend) {
    const int leader = __ffs(pend) - 1;
    const uint32_t gop = __shfl_sync(FULL, exec_op, leader);
    const uint32_t grp = __shfl_sync(FULL, peers, leader);
    if (grp & (1u << lane)) {
      switch (gop) {   // uniform over the group
        case 1u:       // LOD
          r.a = MASKED ? (j & wm) : j;
          break;
        case 2u: {     // ADD
          const uint64_t v = M[jm];
          const uint64_t s = a + v;
          if (CHECKED && (int64_t)((a ^ s) & (v ^ s)) < 0) result = ST_FAULT_OVERFLOW;
          else r.a = MASKED ? (s & wm) : s;
          break;
        }
        case 3u: {     // MUL
          const uint64_t v = M[jm];
          const uint64_t p = a * v;
          if (CHECKED && __mul64hi((long long)a, (long long)v) != ((int64_t)p >> 63)) result = ST_FAULT_OVERFLOW;
          else r.a = MASKED ? (p & wm) : p;
          break;
        }
        case 4u:       // STO
          M[jm] = a;
          break;
        case 5u:       // BNZ
          taken = (a != 0);
          break;
        case 6u:       // RD
          M[jm] = T[r.u0];
          r.u0 += 1u;
          break;
        default: {     // PRI
          const uint64_t v = M[jm];
          if (r.y0 < P.s) {
            Y[r.y0] = v;
            r.y0 += 1u;
          } else if (HIST) {
            h.c[8] += 1u;
          }
          break;
        }
      }
    }
    pend &= ~grp;
  }
  if (exec_op != 0u && result == CONT) {
    if (taken) {
      r.i = j;
      r.ip = jm;
    } else {
      const uint64_t ni = (i + 2ull) & wm;
      uint32_t nip = ip + 2u;
      if (nip >= n) nip -= n;
      if (nip >= n) nip -= n;
      if (ni < i) nip = (ni < n) ? (uint32_t)ni : 0u;
      r.i = ni;
      r.ip = nip;
    }
    r.steps += 1ull;
    if (HIST) {
#pragma unroll
      for (uint32_t k = 1; k <= 7; ++k) h.c[k] += (exec_op == k) ? 1u : 0u;
      h.c[9] += taken ? 1u : 0u;
    }
  }
  return result;
}

// ------------------------------------------------------------------ plain
template <bool MASKED, bool CHECKED, bool HIST, bool VOTE>
__global__ void __launch_bounds__(256) k_plain(DevState S, Params P, const uint32_t* __restrict__ ids,
                                               uint32_t count) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  Hist h;
  h.zero();
  bool active = false;
  uint32_t v = 0;
  Regs r;
  uint64_t* M = nullptr;
  const uint64_t* T = nullptr;
  uint64_t* Y = nullptr;
  if (t < count) {
    v = ids ? ids[t] : t;
    if (S.status[v] == ST_RUNNING) {
      load_regs(S, P, v, r);
      M = S.mem + S.mem_off[v];
      T = S.tape + (uint64_t)v * P.ellp;
      Y = S.y + (uint64_t)v * P.sp;
      active = true;
    }
  }
  uint32_t st = ST_RUNNING;
  if (VOTE) {
    const bool had = active;
    while (__any_sync(FULL, active)) {
      const uint32_t s = vote_step<MASKED, CHECKED, HIST>(M, T, Y, P, r, h, active);
      if (active && s != CONT) {
        st = s;
        active = false;
      }
    }
    if (had) store_regs(S, v, r, st);
  } else if (active) {
    do {
      st = one_step<MASKED, CHECKED, HIST>(M, T, Y, P, r, h);
    } while (st == CONT);
    store_regs(S, v, r, st);
  }
  flush_hist<HIST>(P, h);
}

// ------------------------------------------------------------------ persistent
template <bool MASKED, bool CHECKED, bool HIST, bool VOTE, bool STAGED>
__global__ void __launch_bounds__(256) k_persist(DevState S, Params P, Queue Q, uint32_t ncap,
                                                 uint32_t slot_words, uint32_t epoch, uint32_t refill_min) {
  extern __shared__ __align__(16) uint64_t smem[];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  // per warp: 32 mbarriers (256 B), then 32 lane slots [M | tape | y]
  uint64_t* wbase = smem + (uint64_t)warp * (32u + 32u * slot_words);
  uint64_t* slot = wbase + 32u + (uint64_t)lane * slot_words;
  const uint32_t bar = smem_addr(wbase + lane);
  const uint32_t slot_s = smem_addr(slot);
  uint32_t phase = 0;
  if (STAGED) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncwarp();

  Hist h;
  h.zero();
  Regs r;
  r.i = r.a = r.steps = r.stop = r.cap = 0;
  r.ip = 0; r.n = 1; r.u0 = r.y0 = 0;
  int32_t vm = -1;
  bool active = false, exhausted = false, dead = false;
  uint32_t final_st = ST_RUNNING;
  uint64_t moff = 0;
  uint64_t* M = slot;
  const uint64_t* T = slot;
  uint64_t* Y = slot;
  const uint32_t tbytes = P.ellp * 8u, ybytes = P.sp * 8u;

  for (;;) {
    // ---- claim VMs for lanes that have none (one atomic per warp)
    const bool need = (vm < 0) && !exhausted;
    const uint32_t needm = __ballot_sync(FULL, need);
    if (needm) {
      const int leader = __ffs(needm) - 1;
      uint32_t base = 0;
      if ((int)lane == leader) base = atomicAdd(Q.head, (uint32_t)__popc(needm));
      base = __shfl_sync(FULL, base, leader);
      bool fresh = false;
      if (need) {
        const uint32_t pos = base + (uint32_t)__popc(needm & ((1u << lane) - 1u));
        if (pos < Q.count) {
          const uint32_t cand = Q.ids[pos];
          if (S.status[cand] == ST_RUNNING) {
            vm = (int32_t)cand;
            load_regs(S, P, cand, r);
            moff = S.mem_off[cand];
            fresh = true;
          }
        } else {
          exhausted = true;
        }
      }
      if (fresh) {
        if (STAGED) {
          const uint32_t mbytes = ((r.n + 1u) & ~1u) * 8u;
          mbar_arrive_expect_tx(bar, mbytes + tbytes + ybytes);
          bulk_g2s(slot_s, S.mem + moff, mbytes, bar);
          if (tbytes) bulk_g2s(slot_s + ncap * 8u, S.tape + (uint64_t)vm * P.ellp, tbytes, bar);
          if (ybytes) bulk_g2s(slot_s + (ncap + P.ellp) * 8u, S.y + (uint64_t)vm * P.sp, ybytes, bar);
          M = slot;
          T = slot + ncap;
          Y = slot + ncap + P.ellp;
          if (!mbar_wait_bounded(bar, phase, WAIT_LIMIT)) {
            atomicExch(P.err, ERR_WAIT_TIMEOUT);
            dead = true;          // copies may still land: never touch the slot again
            exhausted = true;
            vm = -1;
            fresh = false;
          }
          phase ^= 1u;
        } else {
          M = S.mem + moff;
          T = S.tape + (uint64_t)vm * P.ellp;
          Y = S.y + (uint64_t)vm * P.sp;
        }
        active = fresh;
      }
    }
    if (__all_sync(FULL, exhausted && !active)) break;
    if (!__any_sync(FULL, active)) continue;

    // ---- run until enough lanes can be refilled (checked every `epoch` steps)
    for (;;) {
      if (VOTE) {
        for (uint32_t t = 0; t < epoch; ++t) {
          const uint32_t s = vote_step<MASKED, CHECKED, HIST>(M, T, Y, P, r, h, active);
          if (active && s != CONT) {
            active = false;
            final_st = s;
          }
        }
      } else {
        for (uint32_t t = 0; t < epoch; ++t) {
          if (active) {
            const uint32_t s = one_step<MASKED, CHECKED, HIST>(M, T, Y, P, r, h);
            if (s != CONT) {
              active = false;
              final_st = s;
            }
          }
        }
      }
      if (!__any_sync(FULL, active)) break;
      const uint32_t want = __ballot_sync(FULL, !active && !exhausted);
      if ((uint32_t)__popc(want) >= refill_min) break;
    }

    // ---- write back lanes whose VM stopped
    if (vm >= 0 && !active) {
      store_regs(S, (uint32_t)vm, r, final_st);
      if (STAGED) {
        fence_proxy_async_smem();
        bulk_s2g(S.mem + moff, slot_s, ((r.n + 1u) & ~1u) * 8u);
        if (ybytes) bulk_s2g(S.y + (uint64_t)vm * P.sp, slot_s + (ncap + P.ellp) * 8u, ybytes);
        bulk_commit();
      }
      vm = -1;
    }
    if (STAGED) bulk_wait_read_all();   // slot reusable once the stores have read it
  }
  if (STAGED) {
    bulk_wait_all();
    if (dead) mbar_wait_bounded(bar, phase ^ 1u, WAIT_LIMIT);   // let stray copies land
  }
  flush_hist<HIST>(P, h);
}

// ------------------------------------------------------------------ stats
__global__ void __launch_bounds__(256) k_stats(DevState S, uint32_t num_vms, unsigned long long* out) {
  unsigned long long steps = 0, c[5] = {0, 0, 0, 0, 0};
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < num_vms; v += gridDim.x * blockDim.x) {
    steps += S.steps[v];
    const uint32_t s = S.status[v];
#pragma unroll
    for (uint32_t k = 0; k < 5; ++k) c[k] += (s == k) ? 1ull : 0ull;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    steps += __shfl_down_sync(FULL, steps, off);
#pragma unroll
    for (int k = 0; k < 5; ++k) c[k] += __shfl_down_sync(FULL, c[k], off);
  }
  if ((threadIdx.x & 31u) == 0) {
    if (steps) atomicAdd(&out[0], steps);
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (c[k]) atomicAdd(&out[1 + k], c[k]);
  }
}

// ------------------------------------------------------------------ launchers
namespace {

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

using PlainFn = void (*)(DevState, Params, const uint32_t*, uint32_t);
using PersistFn = void (*)(DevState, Params, Queue, uint32_t, uint32_t, uint32_t, uint32_t);

template <bool M_, bool C_, bool H_>
PlainFn plain_fn(bool vote) {
  return vote ? k_plain<M_, C_, H_, true> : k_plain<M_, C_, H_, false>;
}

PlainFn pick_plain(const StepVariant& v) {
  if (v.checked) return v.hist ? plain_fn<false, true, true>(v.vote) : plain_fn<false, true, false>(v.vote);
  if (v.masked) return v.hist ? plain_fn<true, false, true>(v.vote) : plain_fn<true, false, false>(v.vote);
  return v.hist ? plain_fn<false, false, true>(v.vote) : plain_fn<false, false, false>(v.vote);
}

template <bool M_, bool C_, bool H_>
PersistFn persist_fn(bool vote, bool staged) {
  if (vote) return staged ? k_persist<M_, C_, H_, true, true> : k_persist<M_, C_, H_, true, false>;
  return staged ? k_persist<M_, C_, H_, false, true> : k_persist<M_, C_, H_, false, false>;
}

PersistFn pick_persist(const StepVariant& v, bool staged) {
  if (v.checked)
    return v.hist ? persist_fn<false, true, true>(v.vote, staged) : persist_fn<false, true, false>(v.vote, staged);
  if (v.masked)
    return v.hist ? persist_fn<true, false, true>(v.vote, staged) : persist_fn<true, false, false>(v.vote, staged);
  return v.hist ? persist_fn<false, false, true>(v.vote, staged) : persist_fn<false, false, false>(v.vote, staged);
}

}  // namespace

cudaError_t launch_pack(const DevState& S, const uint64_t* prog, const uint64_t* prog_off,
                        const uint32_t* prog_of_vm, uint32_t num_vms, uint64_t wmask, uint32_t sp,
                        cudaStream_t stream) {
  if (!num_vms) return cudaSuccess;
  const uint32_t warps_needed = num_vms;
  uint32_t blocks = (warps_needed + 7u) / 8u;
  const uint32_t cap = (uint32_t)num_sms() * 16u;
  if (blocks > cap) blocks = cap;
  k_pack<<<blocks, 256, 0, stream>>>(S, prog, prog_off, prog_of_vm, num_vms, wmask, sp);
  return cudaGetLastError();
}

cudaError_t launch_plain(const StepVariant& var, const DevState& S, const Params& P, const uint32_t* ids,
                         uint32_t count, cudaStream_t stream) {
  if (!count) return cudaSuccess;
  const uint32_t blocks = (count + 255u) / 256u;
  pick_plain(var)<<<blocks, 256, 0, stream>>>(S, P, ids, count);
  return cudaGetLastError();
}

int persist_configure(const StepVariant& var, PersistShape& sh) {
  PersistFn fn = pick_persist(var, sh.staged);
  const size_t per_warp = sh.staged ? (size_t)(32u + 32u * sh.slot_words) * 8u : 0u;
  sh.smem = per_warp * sh.warps;
  if (sh.smem > 48u * 1024u) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)(32u * sh.warps), sh.smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  sh.grid = (uint32_t)(per_sm * num_sms());
  return per_sm;
}

cudaError_t launch_persist(const StepVariant& var, const DevState& S, const Params& P, const Queue& Q,
                           const PersistShape& sh, cudaStream_t stream) {
  if (!Q.count || !sh.grid) return cudaSuccess;
  PersistFn fn = pick_persist(var, sh.staged);
  uint32_t grid = sh.grid;
  const uint32_t lanes_needed = (Q.count + 31u) / 32u;   // warps worth of VMs
  const uint32_t max_useful = (lanes_needed + sh.warps - 1u) / sh.warps;
  if (grid > max_useful) grid = max_useful;
  fn<<<grid, 32u * sh.warps, sh.smem, stream>>>(S, P, Q, sh.ncap, sh.slot_words, sh.epoch, sh.refill_min);
  return cudaGetLastError();
}

cudaError_t launch_stats(const DevState& S, uint32_t num_vms, unsigned long long* out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(out, 0, 6 * sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  if (!num_vms) return cudaSuccess;
  uint32_t blocks = (num_vms + 255u) / 256u;
  const uint32_t cap = (uint32_t)num_sms() * 8u;
  if (blocks > cap) blocks = cap;
  k_stats<<<blocks, 256, 0, stream>>>(S, num_vms, out);
  return cudaGetLastError();
}

}  // namespace rasp
