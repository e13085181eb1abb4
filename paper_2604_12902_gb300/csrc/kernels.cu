// kernels.cu -- sm_103a kernels of the batched word-RASP engine.
//
//   k_pack     c_0(P, x) for every VM (Sec. 2.1): M = P 0^(n-2m), y = 0,
//              i = a = steps = u_0 = y_0 = 0. One warp per chunk of VMs, 16-byte stores.
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
constexpr uint32_t WAIT_LIMIT = 1u << 22;   // mbarrier polls before giving up (default; the
                                           // staged kernel takes its limit as an argument)

// ------------------------------------------------------------------ pack
// Program words as the pack reads them: 8-byte words, or 4-byte words
// (every word of the programs fits in 32 bits) sign-extended to 8 bytes.
__device__ __forceinline__ ulonglong2 prog_pair(const uint64_t* src, uint32_t k) {
  return *reinterpret_cast<const ulonglong2*>(src + k);
}
__device__ __forceinline__ uint64_t prog_word(const uint64_t* src, uint32_t k) { return src[k]; }
__device__ __forceinline__ ulonglong2 prog_pair(const int32_t* src, uint32_t k) {
  const int2 q = *reinterpret_cast<const int2*>(src + k);
  return make_ulonglong2((uint64_t)(int64_t)q.x, (uint64_t)(int64_t)q.y);
}
__device__ __forceinline__ uint64_t prog_word(const int32_t* src, uint32_t k) { return (uint64_t)(int64_t)src[k]; }

// With `lazy` (shared programs on the shared-program schedule) the program
// words M[0, plen) are not written: the steps read them from the program
// itself until the VM writes one of them (see ShView), so only the data
// words are packed.
//
// A warp packs chunks of cl consecutive VMs (cl a power of two <= 32). Each
// lane below cl first fetches the layout of one VM of the chunk (program
// offset and length, n, slab offset) and resets that VM's registers, so
// that the chunk's dependent layout loads take one round trip and the
// register and y stores are coalesced; then the warp writes the chunk's
// slabs one VM at a time, with 16-byte stores.
template <class W>
__global__ void __launch_bounds__(256) k_pack(DevState S, const W* __restrict__ prog,
                                              const uint64_t* __restrict__ prog_off,
                                              const uint32_t* __restrict__ prog_of_vm, uint32_t num_vms,
                                              uint64_t wmask, uint32_t sp, uint32_t lazy, uint32_t cl) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t chunks = (num_vms + cl - 1u) / cl;
  for (uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < chunks; c += warps) {
    const uint32_t v0 = c * cl;
    const uint32_t cnt = min(cl, num_vms - v0);
    const uint32_t v = v0 + lane;
    uint64_t po_l = 0, plen_l = 0, mo_l = 0;
    uint32_t npad_l = 0;
    if (lane < cnt) {
      const uint32_t p = prog_of_vm ? prog_of_vm[v] : v;
      po_l = prog_off[p];
      plen_l = prog_off[p + 1] - po_l;
      npad_l = (S.n[v] + 1u) & ~1u;
      mo_l = S.mem_off[v];
      S.i[v] = 0;
      S.a[v] = 0;
      S.steps[v] = 0;
      S.status[v] = ST_RUNNING;
      S.uhead[v] = 0;
      S.ylen[v] = 0;
      if (S.codedirty) S.codedirty[v] = 0;
    }
    uint64_t* Y = S.y + (uint64_t)v0 * sp;             // the chunk's outputs are one range
    for (uint32_t k = lane; k < cnt * sp; k += 32u) Y[k] = 0ull;
    for (uint32_t j = 0; j < cnt; ++j) {
      const uint64_t po = __shfl_sync(FULL, po_l, j);
      const uint64_t plen = __shfl_sync(FULL, plen_l, j);
      const uint32_t npad = __shfl_sync(FULL, npad_l, j);
      const uint64_t mo = __shfl_sync(FULL, mo_l, j);
      const W* src = prog + po;                        // po is even: pairs are aligned
      if (S.mem32) {
        // narrow batch (w <= 32): 4-byte words, two per 8-byte store
        uint32_t* dst = S.mem32 + mo;
        for (uint32_t k = 2u * lane; k < npad; k += 64u) {
          uint2 w;
          if (k + 1u < plen) {
            const ulonglong2 q = prog_pair(src, k);
            w.x = (uint32_t)(q.x & wmask);
            w.y = (uint32_t)(q.y & wmask);
          } else {
            w.x = (k < plen) ? (uint32_t)(prog_word(src, k) & wmask) : 0u;
            w.y = 0u;
          }
          *reinterpret_cast<uint2*>(dst + k) = w;
        }
        continue;
      }
      uint64_t* dst = S.mem + mo;
      for (uint32_t k = (lazy ? (uint32_t)plen : 0u) + 2u * lane; k < npad; k += 64u) {
        ulonglong2 w;
        if (k + 1u < plen) {
          w = prog_pair(src, k);
          w.x &= wmask;
          w.y &= wmask;
        } else {
          w.x = (k < plen) ? (prog_word(src, k) & wmask) : 0ull;
          w.y = 0ull;
        }
        *reinterpret_cast<ulonglong2*>(dst + k) = w;
      }
    }
  }
}

// ------------------------------------------------------------------ vote step
// Warp-synchronous step: every lane of the warp calls it; `active` lanes
// take part. Lanes are grouped by opcode with __match_any_sync and each group
// runs the handler of its case of the Sec. 2.1 equation. Returns CONT or a
// final status like one_step.
template <bool MASKED, bool CHECKED, bool HIST, class Mem>
__device__ __forceinline__ uint32_t vote_step(Mem M, const uint64_t* __restrict__ T, uint64_t* __restrict__ Y,
                                              const Params& P, Regs& r, Hist& h, bool active) {
  Decoded d;
  d.j = 0;
  d.op = 0;
  d.jm = 0;
  d.jin = false;
  d.taken = false;
  uint32_t result = CONT;
  if (active) result = decode<MASKED, CHECKED>(M, P, r, d);
  const uint32_t exec_op = (active && result == CONT) ? d.op : 0u;
  uint32_t pend = __ballot_sync(FULL, exec_op != 0u);
  const uint32_t peers = __match_any_sync(FULL, exec_op);
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t a = r.a;
  const uint64_t wm = MASKED ? P.wmask : ~0ull;
  while (pend) {
    const int leader = __ffs(pend) - 1;
    const uint32_t gop = __shfl_sync(FULL, exec_op, leader);
    const uint32_t grp = __shfl_sync(FULL, peers, leader);
    if (grp & (1u << lane)) {
      switch (gop) {   // uniform over the group
        case 1u:       // LOD
          r.a = d.j & wm;
          break;
        case 2u: {     // ADD
          const uint64_t v = mem_rd(M, r.clean, d.jm);
          const uint64_t s = a + v;
          if (CHECKED && (int64_t)((a ^ s) & (v ^ s)) < 0) result = ST_FAULT_OVERFLOW;
          else r.a = s & wm;
          break;
        }
        case 3u: {     // MUL
          const uint64_t v = mem_rd(M, r.clean, d.jm);
          const uint64_t p = a * v;
          if (CHECKED && __mul64hi((long long)a, (long long)v) != ((int64_t)p >> 63)) result = ST_FAULT_OVERFLOW;
          else r.a = p & wm;
          break;
        }
        case 4u:       // STO
          mem_wr(M, r.clean, d.jm, a);
          break;
        case 5u:       // BNZ: the jump itself is taken in advance()
          break;
        case 6u:       // RD
          mem_wr(M, r.clean, d.jm, T[r.u0]);
          r.u0 += 1u;
          break;
        default: {     // PRI
          const uint64_t v = mem_rd(M, r.clean, d.jm);
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
    advance<MASKED>(P, r, d);
    count_step<HIST>(h, exec_op, d.taken);
  }
  return result;
}

// ------------------------------------------------------------------ plain
// The memory view of VM v at word offset moff: its slab of 8-byte words, or
// of 4-byte words in a narrow batch.
__device__ __forceinline__ void attach_mem(uint64_t*& M, const DevState& S, uint64_t moff) { M = S.mem + moff; }
__device__ __forceinline__ void attach_mem(NarrowView& M, const DevState& S, uint64_t moff) { M.M = S.mem32 + moff; }

template <bool MASKED, bool CHECKED, bool HIST, bool VOTE, bool CLASSIC = false, bool NARROW = false>
__global__ void __launch_bounds__(256) k_plain(DevState S, Params P, const uint32_t* __restrict__ ids,
                                               uint32_t count) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  Hist h;
  h.zero();
  bool active = false;
  uint32_t v = 0;
  Regs r{};
  std::conditional_t<NARROW, NarrowView, uint64_t*> M{};
  const uint64_t* T = nullptr;
  uint64_t* Y = nullptr;
  if (t < count) {
    v = ids ? ids[t] : t;
    if (S.status[v] == ST_RUNNING) {
      load_regs(S, P, v, r);
      arm_regs(P, r);
      attach_mem(M, S, S.mem_off[v]);
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
      st = one_step<MASKED, CHECKED, HIST, false, CLASSIC>(M, T, Y, P, r, h);
    } while (st == CONT);
    store_regs(S, v, r, st);
  }
  flush_hist<HIST>(P, h);
}

// Run `epoch` steps of every active lane (warp-uniform loop).
template <bool MASKED, bool CHECKED, bool HIST, bool VOTE, bool PIPE, bool CLASSIC = false, class Mem>
__device__ __forceinline__ void run_epoch(Mem M, const uint64_t* T, uint64_t* Y, const Params& P, Regs& r,
                                          Hist& h, bool& active, uint32_t& final_st, uint32_t epoch) {
  if (VOTE) {
    for (uint32_t t = 0; t < epoch; ++t) {
      const uint32_t s = vote_step<MASKED, CHECKED, HIST>(M, T, Y, P, r, h, active);
      if (active && s != CONT) {
        active = false;
        final_st = s;
      }
    }
  } else if (active) {
    for (uint32_t t = 0; t < epoch; ++t) {
      const uint32_t s = one_step<MASKED, CHECKED, HIST, PIPE, CLASSIC>(M, T, Y, P, r, h);
      if (s != CONT) {
        active = false;
        final_st = s;
        break;
      }
    }
  }
}

// Run up to `epoch` steps of every active lane with the epoch loop of
// fast_loop_ptx (WRAP, no counters, select dispatch). Each round runs the
// loop for at most the smallest step countdown of the warp; then the lanes
// whose step needs the general path (the loop left by a warp vote, nothing
// of that step applied) or whose countdown ended take one step with
// step_general, and every active lane re-enters the loop together. A round
// with general steps counts one more step of the epoch, so the epoch always
// ends. With idle_exit > 0 the epoch also ends once that many lanes that were
// running at its start have stopped, so that they are refilled sooner.
template <bool MASKED, bool CLASSIC, class Mem>
__device__ __forceinline__ void run_epoch_loop(Mem M, const uint64_t* T, uint64_t* Y, const Params& P,
                                               Regs& r, Hist& h, bool& active, uint32_t& final_st, uint32_t epoch,
                                               uint32_t idle_exit) {
  const uint32_t mask0 = __ballot_sync(FULL, active);
  uint32_t mask = mask0;
  uint32_t k = epoch;
  while (k && mask) {
    uint32_t done = 0;
    bool general = false;
    if (active) {
      uint32_t kk = min(k, __reduce_min_sync(mask, r.left));
      uint32_t rare = 0;
      if (kk) {
        const uint32_t k0 = kk;
        uint32_t hv = r.have ? 1u : 0u;
        uint64_t co = r.cur.x, cj = r.cur.y;
        if constexpr (std::is_same<Mem, ShView>::value) {
          // clean: code from the shared program (fetch limit min(plen, ilim)),
          // data accesses below plen through the general step
          const bool cl = r.clean;
          rare = fast_loop_ptx_sh<MASKED>(M.M, cl ? M.Pg : M.M, cl ? M.plen : 0u, T, Y, r.n, P.ell, P.s,
                                          cl ? min(M.plen, r.ilim) : r.ilim, P.wmask, mask, r.a, co, cj, r.ip,
                                          r.u0, r.y0, hv, kk);
        } else if constexpr (std::is_same<Mem, NarrowView>::value) {
          // 4-byte words: the loop runs on 32-bit values (w <= 32)
          uint32_t a32 = (uint32_t)r.a, co32 = (uint32_t)co, cj32 = (uint32_t)cj;
          const uint32_t wm32 = (uint32_t)P.wmask;
          if (wm32 == 0xFFFFFFFFu)
            rare = fast_loop_ptx_narrow<false, CLASSIC>(M.M, T, Y, r.n, P.ell, P.s, r.ilim, wm32, mask, a32, co32,
                                                        cj32, r.ip, r.u0, r.y0, hv, kk);
          else
            rare = fast_loop_ptx_narrow<true, CLASSIC>(M.M, T, Y, r.n, P.ell, P.s, r.ilim, wm32, mask, a32, co32,
                                                       cj32, r.ip, r.u0, r.y0, hv, kk);
          r.a = a32;
          co = co32;
          cj = cj32;
        } else if constexpr (std::is_same<Mem, SmemView>::value) {
          // M, tape and y in shared memory: generic addresses, word opcode set
          rare = fast_loop_ptx_gen<MASKED>(M.M, T, Y, r.n, P.ell, P.s, r.ilim, P.wmask, mask, r.a, co, cj, r.ip,
                                           r.u0, r.y0, hv, kk);
        } else {
          rare = fast_loop_ptx<MASKED, CLASSIC>(M, T, Y, r.n, P.ell, P.s, r.ilim, P.wmask, mask, r.a, co, cj, r.ip,
                                                r.u0, r.y0, hv, kk);
        }
        r.cur.x = co;
        r.cur.y = cj;
        r.have = hv != 0u;
        done = k0 - kk;
        r.left -= done;
      }
      general = rare || r.left == 0u;
      if (general) {
        if (r.ip >= r.ilim) {
          // the loop took i (+) 2 = ip + 2 unreduced (ibase = 0): reduce it
          const uint64_t i = (uint64_t)r.ip & P.wmask;
          r.ip = mod_n(i, r.n);
          r.ibase = i - r.ip;
        }
        r.have = false;
        const uint32_t st = step_general<MASKED, false, false, CLASSIC>(M, T, Y, P, r, h);
        if (st == CONT) {
          prime(M, r);
        } else {
          active = false;
          final_st = st;
        }
      }
    }
    done = __shfl_sync(FULL, done, __ffs(mask) - 1);        // the same in every lane of the mask
    k -= done;
    if (__any_sync(FULL, general) && k) k -= 1u;
    mask = __ballot_sync(FULL, active);
    if (idle_exit && (uint32_t)__popc(mask0 & ~mask) >= idle_exit) break;
  }
}

// ------------------------------------------------------------------ persistent, staged in SMEM
template <bool MASKED, bool CHECKED, bool HIST, bool VOTE, bool LOOP = false>
__global__ void __launch_bounds__(256) k_persist(DevState S, Params P, Queue Q, uint32_t ncap,
                                                 uint32_t slot_words, uint32_t epoch, uint32_t refill_min,
                                                 uint32_t wait_limit) {
  extern __shared__ __align__(16) uint64_t smem[];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  // per warp: 32 mbarriers (256 B), then 32 lane slots [M | tape | y]
  uint64_t* wbase = smem + (uint64_t)warp * (32u + 32u * slot_words);
  uint64_t* slot = wbase + 32u + (uint64_t)lane * slot_words;
  const uint32_t bar = smem_addr(wbase + lane);
  const uint32_t slot_s = smem_addr(slot);
  uint32_t phase = 0;
  mbar_init(bar, 1);
  fence_mbar_init();
  __syncwarp();

  Hist h;
  h.zero();
  Regs r{};
  r.n = 1;
  int32_t vm = -1;
  bool active = false, exhausted = false, dead = false;
  uint32_t final_st = ST_RUNNING;
  uint64_t moff = 0;
  uint64_t* M = slot;
  const uint64_t* T = slot + ncap;
  uint64_t* Y = slot + ncap + P.ellp;
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
      if (fresh && ((r.n + 1u) & ~1u) > ncap) {
        // the VM does not fit this bucket's slot: refuse it (flag, not a copy past the slot)
        atomicExch(P.err, ERR_SLOT);
        vm = -1;
        fresh = false;
      }
      if (fresh) {
        arm_regs(P, r);
        const uint32_t mbytes = ((r.n + 1u) & ~1u) * 8u;
        mbar_arrive_expect_tx(bar, mbytes + tbytes + ybytes);
        bulk_g2s(slot_s, S.mem + moff, mbytes, bar);
        if (tbytes) bulk_g2s(slot_s + ncap * 8u, S.tape + (uint64_t)vm * P.ellp, tbytes, bar);
        if (ybytes) bulk_g2s(slot_s + (ncap + P.ellp) * 8u, S.y + (uint64_t)vm * P.sp, ybytes, bar);
        if (!mbar_wait_bounded(bar, phase, wait_limit)) {
          atomicExch(P.err, ERR_WAIT_TIMEOUT);
          dead = true;          // copies may still land: never touch the slot again
          exhausted = true;
          vm = -1;
          fresh = false;
        }
        phase ^= 1u;
        active = fresh;
        if (LOOP && fresh) prime(M, r);
      }
    }
    if (__all_sync(FULL, exhausted && !active)) break;
    if (!__any_sync(FULL, active)) continue;

    // ---- run until enough lanes can be refilled (checked every `epoch` steps)
    for (;;) {
      if constexpr (LOOP)
        run_epoch_loop<MASKED, false>(SmemView{M}, T, Y, P, r, h, active, final_st, epoch, 0u);
      else
        run_epoch<MASKED, CHECKED, HIST, VOTE, false>(M, T, Y, P, r, h, active, final_st, epoch);
      if (!__any_sync(FULL, active)) break;
      const uint32_t want = __ballot_sync(FULL, !active && !exhausted);
      if ((uint32_t)__popc(want) >= refill_min) break;
    }

    // ---- write back lanes whose VM stopped
    if (vm >= 0 && !active) {
      store_regs(S, (uint32_t)vm, r, final_st);
      fence_proxy_async_smem();
      bulk_s2g(S.mem + moff, slot_s, ((r.n + 1u) & ~1u) * 8u);
      if (ybytes) bulk_s2g(S.y + (uint64_t)vm * P.sp, slot_s + (ncap + P.ellp) * 8u, ybytes);
      bulk_commit();
      vm = -1;
    }
    bulk_wait_read_all();   // slot reusable once the stores have read it
  }
  bulk_wait_all();
  if (dead) mbar_wait_bounded(bar, phase ^ 1u, WAIT_LIMIT);   // let stray copies land
  flush_hist<HIST>(P, h);
}

// ------------------------------------------------------------------ persistent, M in HBM
// Each lane runs one VM at a time with M, tape and y in HBM (cached in L1).
// The next VM of every lane is prefetched in stages that overlap the
// running VM -- queue position, VM id (ids[pos]), then its state-store
// entries warmed into L2 -- so a lane whose VM stops swaps the next one in
// with one L2 round trip. (Holding the next VM's registers instead cost ~14
// live registers in the step loop and forced spills.) Queue
// positions below Q.soft_end are claimed in warp chunks of 32, the next
// chunk's atomic issued while the current one is still being used. The
// last positions (as many as there are resident lanes) form the tail: they
// are claimed one at a time, only by lanes that are idle, so that near the
// end no VM waits in a busy lane's prefetch slot while other lanes idle.
enum : uint32_t { PF_EMPTY = 0, PF_ID = 1, PF_REGS = 2, PF_NONE = 3 };   // PF_REGS: entries warmed in L2

template <bool MASKED, bool CHECKED, bool HIST, bool VOTE, bool CLASSIC = false, bool LOOP = false,
          bool NARROW = false>
__global__ void __launch_bounds__(128, 7) k_persist_gl(DevState S, Params P, Queue Q, uint32_t epoch,
                                                       uint32_t idle_exit) {
  static_assert(!LOOP || (!CHECKED && !HIST && !VOTE), "the epoch loop serves WRAP select steps without counters");
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  Hist h;
  h.zero();
  // A compacted queue (budget rounds): its length is read on the device, and
  // the first chunk of every warp is assigned statically, interleaved across
  // CTAs (warp w of CTA c takes chunk w * gridDim.x + c), so that a queue
  // shorter than the resident lanes is spread evenly over the SMs instead of
  // going to whichever warps win the first atomics. Later chunks are claimed
  // dynamically past the statically assigned ones; there is no one-at-a-time
  // tail phase.
  const bool stat = Q.dcount != nullptr;
  const uint32_t claim_off = stat ? gridDim.x * blockDim.x : 0u;
  if (stat) {
    Q.count = *Q.dcount;
    Q.soft_end = Q.count;
  }
  // warp chunk [cpos, cend) of main-phase queue positions
  uint32_t tick = 0;
  if (stat) tick = (((uint32_t)threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32u;
  else if (lane == 0) tick = atomicAdd(Q.head, 32u);
  uint32_t cpos = __shfl_sync(FULL, tick, 0);
  uint32_t cend = cpos < Q.soft_end ? min(cpos + 32u, Q.soft_end) : cpos;
  bool tail = cpos >= Q.soft_end;  // warp-uniform: main positions used up
  bool inflight = false;           // lane 0 holds the next chunk's ticket in `tick`

  // running VM
  Regs r{};
  r.n = 1;
  int32_t vm = -1;
  bool active = false;
  uint32_t final_st = ST_RUNNING;
  std::conditional_t<NARROW, NarrowView, uint64_t*> M{};
  attach_mem(M, S, 0ull);
  const uint64_t* T = S.tape;
  uint64_t* Y = S.y;
  // prefetched VM
  uint32_t pf = PF_EMPTY, pf_pos = 0, pf_vm = 0;

  for (;;) {
    // ---- boundary: retire stopped VMs
    if (vm >= 0 && !active) {
      store_regs(S, (uint32_t)vm, r, final_st);
      vm = -1;
    }
    // swap in the prefetched VM (its loads were issued a boundary ago)
    if (vm < 0 && pf == PF_REGS) {
      if (S.status[pf_vm] == ST_RUNNING) {
        load_regs(S, P, pf_vm, r);
        const uint64_t moff = S.mem_off[pf_vm];
        arm_regs(P, r);
        vm = (int32_t)pf_vm;
        attach_mem(M, S, moff);
        T = S.tape + (uint64_t)pf_vm * P.ellp;
        Y = S.y + (uint64_t)pf_vm * P.sp;
        if (!VOTE) prime(M, r);
        active = true;
      }
      pf = PF_EMPTY;
    }
    // advance the prefetch pipeline: id -> the VM's entries warmed in L2
    if (pf == PF_ID) {         // pf_vm = ids[pf_pos] was issued a boundary ago
      asm volatile("prefetch.global.L2 [%0];" :: "l"(S.status + pf_vm));
      asm volatile("prefetch.global.L2 [%0];" :: "l"(S.i + pf_vm));
      asm volatile("prefetch.global.L2 [%0];" :: "l"(S.a + pf_vm));
      asm volatile("prefetch.global.L2 [%0];" :: "l"(S.steps + pf_vm));
      asm volatile("prefetch.global.L2 [%0];" :: "l"(S.cap + pf_vm));
      asm volatile("prefetch.global.L2 [%0];" :: "l"(S.n + pf_vm));
      asm volatile("prefetch.global.L2 [%0];" :: "l"(S.uhead + pf_vm));
      asm volatile("prefetch.global.L2 [%0];" :: "l"(S.ylen + pf_vm));
      asm volatile("prefetch.global.L2 [%0];" :: "l"(S.mem_off + pf_vm));
      pf = PF_REGS;
    }
    // ---- new queue positions
    if (!tail) {
      uint32_t needm = __ballot_sync(FULL, pf == PF_EMPTY);
      while (needm && !tail) {
        const uint32_t avail = cend - cpos;
        const uint32_t rank = (uint32_t)__popc(needm & lt);
        if (((needm >> lane) & 1u) && rank < avail) {
          pf_pos = cpos + rank;
          pf = PF_ID;
        }
        const uint32_t took = min((uint32_t)__popc(needm), avail);
        cpos += took;
        needm = __ballot_sync(FULL, pf == PF_EMPTY);
        if (cpos >= cend) {      // chunk used up: take the next one
          if (!inflight && lane == 0) tick = claim_off + atomicAdd(Q.head, 32u);
          inflight = false;
          cpos = __shfl_sync(FULL, tick, 0);
          if (cpos >= Q.soft_end) {
            tail = true;
            cend = cpos;
          } else {
            cend = min(cpos + 32u, Q.soft_end);
          }
        }
      }
      // claim the next chunk early so its atomic is in flight while this one drains
      if (!tail && !inflight && cend - cpos <= 16u && cend < Q.soft_end) {
        if (lane == 0) tick = claim_off + atomicAdd(Q.head, 32u);
        inflight = true;
      }
    }
    if (tail) {
      const uint32_t needm = __ballot_sync(FULL, pf == PF_EMPTY && vm < 0);
      if (needm) {
        const int leader = __ffs(needm) - 1;
        uint32_t base = 0;
        if ((int)lane == leader) base = atomicAdd(Q.tail_head, (uint32_t)__popc(needm));
        base = __shfl_sync(FULL, base, leader);
        if ((needm >> lane) & 1u) {
          const uint32_t pos = Q.soft_end + base + (uint32_t)__popc(needm & lt);
          if (pos < Q.count) {
            pf_pos = pos;
            pf = PF_ID;
          } else {
            pf = PF_NONE;        // queue exhausted for this lane
          }
        }
      }
    }
    if (pf == PF_ID) pf_vm = Q.ids[pf_pos];     // issue the id load; consumed next boundary
    if (tail && vm < 0 && pf == PF_ID) {
      // an idle lane in the tail starts its VM at once (waiting on the loads
      // here) instead of two boundaries later
      pf = PF_EMPTY;
      if (S.status[pf_vm] == ST_RUNNING) {
        load_regs(S, P, pf_vm, r);
        const uint64_t moff = S.mem_off[pf_vm];
        arm_regs(P, r);
        vm = (int32_t)pf_vm;
        attach_mem(M, S, moff);
        T = S.tape + (uint64_t)pf_vm * P.ellp;
        Y = S.y + (uint64_t)pf_vm * P.sp;
        if (!VOTE) prime(M, r);
        active = true;
      }
    }
    // done when no lane runs a VM or has one coming
    if (__all_sync(FULL, vm < 0 && pf == PF_NONE)) break;

    // ---- run
    if constexpr (LOOP) run_epoch_loop<MASKED, CLASSIC>(M, T, Y, P, r, h, active, final_st, epoch, idle_exit);
    else run_epoch<MASKED, CHECKED, HIST, VOTE, true, CLASSIC>(M, T, Y, P, r, h, active, final_st, epoch);
  }
  flush_hist<HIST>(P, h);
}

// ------------------------------------------------------------------ serving: one kernel over a shared ring
// Persistent warps over the ring of VMs of every admitted request (continuous
// batching). Each ring entry names a request slot and a VM of that request's
// batch; lanes claim entries for themselves (two or three atomic adds per
// warp, never past the entries the host has published, so no lane waits for
// work that is not there and nobody retries), run the VM with the same step as the batch kernels, store it
// back and count it off its request. The lane that stops a request's last VM
// writes the request's completion word in host-mapped memory.
//
// The instance lives as a whole: *state counts the warps that hold or are
// claiming work. A warp with nothing to run and an empty ring leaves that
// count and polls; to take work again it rejoins first. When the count is
// zero, an idle warp may close the instance (compare-and-swap 0 -> CLOSING)
// -- at once when the host has launched a newer instance (ordered after every
// later publish), else after idle_polls polls of an empty ring, up to 16 us
// apart --
// and every warp that sees CLOSING returns. So warps never leave while others
// of the instance still run work (the next instance cannot start until this
// one has returned), and nothing waits on the host without a limit.
constexpr unsigned long long SERVE_CLOSING = 1ull << 63;
constexpr uint32_t kServeIdleCeiling = 1u << 16;   // about 1 s of idle polls: the warp leaves, whatever the count says

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// A VM of request `slot` has stopped and its state is stored: count it off.
__device__ __forceinline__ void serve_finish(const ServeArgs& A, uint32_t slot) {
  __threadfence();                                  // the VM's state before the count
  if (atomicSub(&A.pending[slot], 1u) == 1u) {
    __threadfence_system();                         // every VM's state before the completion word
    *reinterpret_cast<volatile uint32_t*>(&A.done[slot]) = A.slots[slot].gen;
  }
}

template <bool MASKED, bool CHECKED, bool CLASSIC>
__global__ void __launch_bounds__(128, 6) k_serve(ServeArgs A, Params P0) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  Hist h;
  h.zero();
  Params P = P0;                 // per lane: P.budget is the running request's
  Regs r{};
  r.n = 1;
  int32_t slot = -1;
  uint32_t vm = 0;
  bool active = false;
  uint32_t final_st = ST_RUNNING;
  uint64_t* M = nullptr;
  const uint64_t* T = nullptr;
  uint64_t* Y = nullptr;
  uint32_t idle = 0;
  bool busy = false;             // warp-uniform: this warp is counted in *A.state
  for (;;) {
    // ---- retire a stopped VM
    if (slot >= 0 && !active) {
      store_regs(A.slots[slot].S, vm, r, final_st);
      serve_finish(A, (uint32_t)slot);
      slot = -1;
    }
    // ---- claim ring positions for the idle lanes: take credits (published,
    // unclaimed entries; a shortfall is given back, so nobody retries), then
    // positions below the published ones with one add on the head
    const uint32_t need = __ballot_sync(FULL, slot < 0);
    uint32_t got = 0;
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      int closing = 0;
      if ((int)lane == leader) {
        const long long c = *reinterpret_cast<volatile long long*>(A.credits);
        if (c > 0) {
          if (!busy) {                            // rejoin before taking work
            if (atomicAdd(A.state, 1ull) & SERVE_CLOSING) closing = 1;
            else busy = true;                     // counted: leaves the count only through the idle path
          }
          if (!closing) {
            const long long want = __popc(need);
            const long long old = (long long)atomicAdd(A.credits, (unsigned long long)(-want));
            const long long g = old >= want ? want : (old > 0 ? old : 0);
            if (g < want) atomicAdd(A.credits, (unsigned long long)(want - g));
            if (g > 0) {
              base = atomicAdd(A.head, (unsigned long long)g);
              got = (uint32_t)g;
            }
            __threadfence();                      // the entries published before the credits, then read
          }
        }
      }
      if (__shfl_sync(FULL, closing, leader)) break;
      busy = __shfl_sync(FULL, busy ? 1 : 0, leader) != 0;
      __syncwarp();
      got = __shfl_sync(FULL, got, leader);
      base = __shfl_sync(FULL, base, leader);
      const uint32_t rank = (uint32_t)__popc(need & lt);
      if (((need >> lane) & 1u) && rank < got) {
        const uint64_t e = A.ring[(base + rank) & A.ring_mask];
        const uint32_t sl = (uint32_t)(e >> 32), v = (uint32_t)e;
        if (sl >= A.num_slots || v >= A.slots[sl].num_vms) {
          atomicExch(A.err, ERR_RING);          // never touch memory an entry does not own
        } else {
          const ServeSlot& sd = A.slots[sl];
          slot = (int32_t)sl;
          vm = v;
          if (sd.S.status[v] == ST_RUNNING) {
            P.budget = sd.budget;
            load_regs(sd.S, P, v, r);
            const uint64_t moff = sd.S.mem_off[v];
            arm_regs(P, r);
            M = sd.S.mem + moff;
            T = sd.S.tape + (uint64_t)v * P.ellp;
            Y = sd.S.y + (uint64_t)v * P.sp;
            if (!CHECKED) prime(M, r);
            active = true;
          } else {
            serve_finish(A, sl);                // already stopped: nothing to run
            slot = -1;
          }
        }
      }
    }
    if (!__any_sync(FULL, active)) {
      if (got == 0 && __all_sync(FULL, slot < 0)) {
        // nothing to run: leave the busy count; close the instance when no
        // warp is busy and (a newer instance exists or the idle polls ran out)
        // (host-mapped words are read only when the count is empty; idle
        // warps back off from 1 to 16 us so that they do not crowd the
        // counters the working warps use)
        int leave = 0;
        if (lane == 0) {
          if (busy) atomicAdd(A.state, ~0ull);       // minus one
          const unsigned long long st = *reinterpret_cast<volatile unsigned long long*>(A.state);
          if (st & SERVE_CLOSING) {
            leave = 1;
          } else if (st == 0ull && (idle + 1u > A.idle_polls || *A.launched > A.instance)) {
            const unsigned long long prev = atomicCAS(A.state, 0ull, SERVE_CLOSING);
            leave = (prev == 0ull || (prev & SERVE_CLOSING)) ? 1 : 0;
          } else if (idle > kServeIdleCeiling) {
            leave = 1;                            // idle this long: this warp leaves (the rest still serve)
          }
        }
        busy = false;
        if (__shfl_sync(FULL, leave, 0)) break;
        __nanosleep(1000u << min(idle, 4u));
        ++idle;
      }
      continue;
    }
    idle = 0;
    // ---- run an epoch
    if constexpr (CHECKED) {
      run_epoch<MASKED, true, false, false, false, CLASSIC>(M, T, Y, P, r, h, active, final_st, A.epoch);
    } else {
      run_epoch_loop<MASKED, CLASSIC>(M, T, Y, P, r, h, active, final_st, A.epoch, 0u);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_system();
    atomicAdd(A.exited, 1u);     // host-mapped: this instance's blocks are done when all have added
  }
}

__global__ void k_ring_fill(uint64_t* __restrict__ ring, uint64_t mask, unsigned long long start, uint32_t slot,
                            const uint32_t* __restrict__ ids, uint32_t count) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x)
    ring[(start + k) & mask] = ((uint64_t)slot << 32) | (uint64_t)(ids ? ids[k] : k);
}

__global__ void k_ring_publish(unsigned long long* credits, unsigned long long count) {
  __threadfence();
  atomicAdd(credits, count);
}

// ------------------------------------------------------------------ shared programs
// One CTA per program (grid-stride over programs): the program's words sit
// once in shared memory and the CTA's lanes run that program's VMs. Each VM
// sees its memory through a shared-program view (ShView): code and other
// program words come from the shared copy while the VM has not written into
// them (Regs::clean), data from the VM's own slab, whose program words
// need not have been written at c_0 (lazy pack); a VM's first write into its
// program words copies the program into its slab. codedirty[v] records that
// the VM's slab holds its own program words.
//
// k_shared: each lane takes the next VM from a shared-memory counter when
// its VM stops and steps it with one_step (CHECKED semantics, counters).
template <bool MASKED, bool CHECKED, bool HIST>
__global__ void __launch_bounds__(128) k_shared(DevState S, Params P, const uint64_t* __restrict__ prog,
                                                const uint64_t* __restrict__ prog_off,
                                                const uint32_t* __restrict__ pv_off,
                                                const uint32_t* __restrict__ pv_ids, uint32_t num_programs,
                                                uint32_t epoch) {
  extern __shared__ __align__(16) uint64_t ps[];
  __shared__ uint32_t next;
  Hist h;
  h.zero();
  for (uint32_t p = blockIdx.x; p < num_programs; p += gridDim.x) {
    const uint64_t po = prog_off[p];
    const uint32_t plen = (uint32_t)(prog_off[p + 1] - po);
    for (uint32_t k = threadIdx.x; k < plen; k += blockDim.x) ps[k] = prog[po + k] & P.wmask;
    if (threadIdx.x == 0) next = 0;
    __syncthreads();
    const uint32_t first = pv_off[p], count = pv_off[p + 1] - first;
    Regs r{};
    r.n = 1;
    int32_t vm = -1;
    uint32_t st = CONT;
    ShView V{S.mem, ps, plen};
    const uint64_t* T = S.tape;
    uint64_t* Y = S.y;
    bool more = true;
    for (;;) {
      if (vm < 0 && more) {
        const uint32_t idx = atomicAdd(&next, 1u);
        if (idx < count) {
          const uint32_t v = pv_ids[first + idx];
          if (S.status[v] == ST_RUNNING) {
            load_regs(S, P, v, r);
            arm_regs(P, r);
            r.clean = S.codedirty[v] == 0;
            V.M = S.mem + S.mem_off[v];
            T = S.tape + (uint64_t)v * P.ellp;
            Y = S.y + (uint64_t)v * P.sp;
            vm = (int32_t)v;
          }
        } else {
          more = false;
        }
      }
      if (vm < 0) {
        if (!more) break;
        continue;
      }
      st = one_step<MASKED, CHECKED, HIST, false>(V, T, Y, P, r, h);
      if (st != CONT) {
        store_regs(S, (uint32_t)vm, r, st);
        if (!r.clean) S.codedirty[vm] = 1;
        vm = -1;
      }
    }
    __syncthreads();   // every lane done with this program's copy
  }
  flush_hist<HIST>(P, h);
}

// k_shared_loop (WRAP, no counters): the lanes of a warp run their VMs in
// epochs of the PTX epoch loop (fast_loop_ptx_sh: instruction pairs of a
// clean VM loaded from the shared copy); at each epoch boundary the lanes
// whose VM stopped store it and take the next VMs of the program (one
// shared-memory atomic per warp).
template <bool MASKED>
__global__ void __launch_bounds__(128, 7) k_shared_loop(DevState S, Params P, const uint64_t* __restrict__ prog,
                                                        const uint64_t* __restrict__ prog_off,
                                                        const uint32_t* __restrict__ pv_off,
                                                        const uint32_t* __restrict__ pv_ids, uint32_t num_programs,
                                                        uint32_t epoch) {
  extern __shared__ __align__(16) uint64_t ps[];
  __shared__ uint32_t next;
  const uint32_t lane = threadIdx.x & 31u;
  Hist h;
  h.zero();
  for (uint32_t p = blockIdx.x; p < num_programs; p += gridDim.x) {
    const uint64_t po = prog_off[p];
    const uint32_t plen = (uint32_t)(prog_off[p + 1] - po);
    for (uint32_t k = threadIdx.x; k < plen; k += blockDim.x) ps[k] = prog[po + k] & P.wmask;
    if (threadIdx.x == 0) next = 0;
    __syncthreads();
    const uint32_t first = pv_off[p], count = pv_off[p + 1] - first;
    Regs r{};
    r.n = 1;
    int32_t vm = -1;
    bool active = false, more = true;
    uint32_t final_st = ST_RUNNING;
    ShView V{S.mem, ps, plen};
    const uint64_t* T = S.tape;
    uint64_t* Y = S.y;
    for (;;) {
      // boundary: retire stopped VMs, then refill idle lanes
      if (vm >= 0 && !active) {
        store_regs(S, (uint32_t)vm, r, final_st);
        if (!r.clean) S.codedirty[vm] = 1;
        vm = -1;
      }
      const uint32_t needm = __ballot_sync(FULL, vm < 0 && more);
      if (needm) {
        const int leader = __ffs(needm) - 1;
        uint32_t base = 0;
        if ((int)lane == leader) base = atomicAdd(&next, (uint32_t)__popc(needm));
        base = __shfl_sync(FULL, base, leader);
        if ((needm >> lane) & 1u) {
          const uint32_t idx = base + (uint32_t)__popc(needm & ((1u << lane) - 1u));
          if (idx < count) {
            const uint32_t v = pv_ids[first + idx];
            if (S.status[v] == ST_RUNNING) {
              load_regs(S, P, v, r);
              arm_regs(P, r);
              r.clean = S.codedirty[v] == 0;
              V.M = S.mem + S.mem_off[v];
              T = S.tape + (uint64_t)v * P.ellp;
              Y = S.y + (uint64_t)v * P.sp;
              vm = (int32_t)v;
              prime(V, r);
              active = true;
            }
          } else {
            more = false;
          }
        }
      }
      if (__all_sync(FULL, vm < 0 && !more)) break;
      if (!__any_sync(FULL, active)) continue;
      run_epoch_loop<MASKED, false>(V, T, Y, P, r, h, active, final_st, epoch, 0u);
    }
    __syncthreads();   // every lane done with this program's copy
  }
}

// The program words of every VM whose slab does not hold them yet (clean VMs
// of a lazily packed shared-program batch): M[0, plen) = P, one warp per VM,
// 16-byte stores.
__global__ void __launch_bounds__(256) k_materialize(DevState S, const uint64_t* __restrict__ prog,
                                                     const uint64_t* __restrict__ prog_off,
                                                     const uint32_t* __restrict__ prog_of_vm, uint32_t num_vms,
                                                     uint64_t wmask) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < num_vms; v += warps) {
    if (S.codedirty[v]) continue;
    const uint32_t p = prog_of_vm ? prog_of_vm[v] : v;
    const uint64_t po = prog_off[p];
    const uint32_t plen = (uint32_t)(prog_off[p + 1] - po);
    const uint64_t* src = prog + po;
    uint64_t* dst = S.mem + S.mem_off[v];
    for (uint32_t k = 2u * lane; k < plen; k += 64u) {
      ulonglong2 w = *reinterpret_cast<const ulonglong2*>(src + k);
      w.x &= wmask;
      w.y &= wmask;
      *reinterpret_cast<ulonglong2*>(dst + k) = w;
    }
  }
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

// ------------------------------------------------------------------ compaction between budget rounds
// The ids of the VMs at positions [0, count) of `ids` whose status is still
// RUNNING, written densely to out[0 .. *out_count) (warp-aggregated; order
// within the output is not specified). *out_count must be zero on entry.
__global__ void __launch_bounds__(256) k_compact(const uint32_t* __restrict__ ids, uint32_t count,
                                                 const uint8_t* __restrict__ status, uint32_t* __restrict__ out,
                                                 uint32_t* __restrict__ out_count) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < count; base += stride) {
    const uint32_t q = base + threadIdx.x;
    uint32_t v = 0;
    bool run = false;
    if (q < count) {
      v = ids[q];
      run = status[v] == ST_RUNNING;
    }
    const uint32_t m = __ballot_sync(FULL, run);
    uint32_t first = 0;
    if (lane == 0 && m) first = atomicAdd(out_count, (uint32_t)__popc(m));
    first = __shfl_sync(FULL, first, 0);
    if (run) out[first + __popc(m & ((1u << lane) - 1u))] = v;
  }
}

// ------------------------------------------------------------------ halting-time histogram
// Sec. 3 (Fig. 1b): the distribution of tau_h, the number of steps after
// which a machine reached its fixed point, over the HALTED machines of the
// batch. counts[k] += number of HALTED VMs with edges[k] <= steps < edges[k+1];
// other[0..3] += RUNNING, TIMEOUT, faulted (either kind), and HALTED VMs
// outside [edges[0], edges[nbins]). Per-block shared-memory counters, one
// global atomic per non-empty bin per block.
__global__ void __launch_bounds__(256) k_tau_hist(const uint64_t* __restrict__ steps,
                                                  const uint8_t* __restrict__ status, uint32_t num_vms,
                                                  const uint64_t* __restrict__ edges, uint32_t nbins,
                                                  unsigned long long* __restrict__ counts,
                                                  unsigned long long* __restrict__ other) {
  extern __shared__ __align__(16) uint64_t se[];       // nbins + 1 edges, then nbins u32 counters
  uint32_t* sc = reinterpret_cast<uint32_t*>(se + nbins + 1);
  __shared__ uint32_t so[4];
  for (uint32_t k = threadIdx.x; k <= nbins; k += blockDim.x) se[k] = edges[k];
  for (uint32_t k = threadIdx.x; k < nbins; k += blockDim.x) sc[k] = 0u;
  if (threadIdx.x < 4) so[threadIdx.x] = 0u;
  __syncthreads();
  const uint64_t lo = se[0], hi = se[nbins];
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < num_vms; v += gridDim.x * blockDim.x) {
    const uint32_t st = status[v];
    if (st == ST_HALTED) {
      const uint64_t t = steps[v];
      if (t < lo || t >= hi) {
        atomicAdd(&so[3], 1u);
      } else {
        uint32_t a = 0, b = nbins;                      // se[a] <= t < se[b]
        while (b - a > 1u) {
          const uint32_t m = (a + b) >> 1;
          if (se[m] <= t) a = m;
          else b = m;
        }
        atomicAdd(&sc[a], 1u);
      }
    } else {
      atomicAdd(&so[st == ST_RUNNING ? 0 : (st == ST_TIMEOUT ? 1 : 2)], 1u);
    }
  }
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < nbins; k += blockDim.x)
    if (sc[k]) atomicAdd(&counts[k], (unsigned long long)sc[k]);
  if (threadIdx.x < 4 && so[threadIdx.x]) atomicAdd(&other[threadIdx.x], (unsigned long long)so[threadIdx.x]);
}

// ------------------------------------------------------------------ top-k halting times
// The k HALTED VMs with the largest tau_h (ties: smaller VM id first), for
// the generate -> run -> filter search loop. Each block keeps a running
// top-k in shared memory: per tile it appends (TILE - k) new candidates
// behind its current best k and bitonic-sorts the TILE entries, so the first
// k are the best of both; blocks write their k to a candidate array, which
// one block reduces the same way.
constexpr uint32_t TOPK_TILE = 2048;

__device__ __forceinline__ bool topk_better(const TopCand& x, const TopCand& y) {
  if (x.ok != y.ok) return x.ok > y.ok;
  if (x.steps != y.steps) return x.steps > y.steps;
  return x.vm < y.vm;
}

// items: VMs [0, count) read from steps/status (cands == NULL), or `count`
// candidates from an earlier pass. out: k candidates per block.
__global__ void __launch_bounds__(1024) k_topk(const uint64_t* __restrict__ steps, const uint8_t* __restrict__ status,
                                               const TopCand* __restrict__ cands, uint32_t count, uint32_t k,
                                               TopCand* __restrict__ out) {
  __shared__ TopCand buf[TOPK_TILE];
  const uint32_t t = threadIdx.x;
  for (uint32_t q = t; q < TOPK_TILE; q += blockDim.x) buf[q] = TopCand{0ull, 0xFFFFFFFFu, 0u};
  __syncthreads();
  const uint32_t fresh = TOPK_TILE - k;
  for (uint64_t base = (uint64_t)blockIdx.x * fresh; base < count; base += (uint64_t)gridDim.x * fresh) {
    for (uint32_t q = t; q < fresh; q += blockDim.x) {
      const uint64_t idx = base + q;
      TopCand c{0ull, 0xFFFFFFFFu, 0u};
      if (idx < count) {
        if (cands) {
          c = cands[idx];
        } else if (status[idx] == ST_HALTED) {
          c = TopCand{steps[idx], (uint32_t)idx, 1u};
        }
      }
      buf[k + q] = c;
    }
    __syncthreads();
    // bitonic sort of buf, best first
    for (uint32_t size = 2; size <= TOPK_TILE; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t q = t; q < TOPK_TILE / 2; q += blockDim.x) {
          const uint32_t lo = 2 * q - (q & (stride - 1));
          const uint32_t hi = lo + stride;
          const bool down = (lo & size) == 0;          // this run sorts best first
          const TopCand x = buf[lo], y = buf[hi];
          if (topk_better(y, x) == down) {
            buf[lo] = y;
            buf[hi] = x;
          }
        }
        __syncthreads();
      }
    }
  }
  for (uint32_t q = t; q < k; q += blockDim.x) out[(uint64_t)blockIdx.x * k + q] = buf[q];
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
using StagedFn = void (*)(DevState, Params, Queue, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t);
using GlobalFn = void (*)(DevState, Params, Queue, uint32_t, uint32_t);

template <bool M_, bool C_, bool H_>
PlainFn plain_fn(bool vote) {
  return vote ? k_plain<M_, C_, H_, true> : k_plain<M_, C_, H_, false>;
}

// The classic opcode set (Sec. 1.1) is built for the select dispatch only.
template <bool CL>
PlainFn plain_select(const StepVariant& v) {
  if (v.narrow) return v.hist ? k_plain<true, false, true, false, CL, true> : k_plain<true, false, false, false, CL, true>;
  if (v.checked) return v.hist ? k_plain<false, true, true, false, CL> : k_plain<false, true, false, false, CL>;
  if (v.masked) return v.hist ? k_plain<true, false, true, false, CL> : k_plain<true, false, false, false, CL>;
  return v.hist ? k_plain<false, false, true, false, CL> : k_plain<false, false, false, false, CL>;
}

template <bool CL>
GlobalFn global_select(const StepVariant& v) {
  if (v.narrow) {
    if (v.hist) return k_persist_gl<true, false, true, false, CL, false, true>;
    if (v.block) return k_persist_gl<true, false, false, false, CL, false, true>;
    return k_persist_gl<true, false, false, false, CL, true, true>;
  }
  if (v.checked)
    return v.hist ? k_persist_gl<false, true, true, false, CL> : k_persist_gl<false, true, false, false, CL>;
  if (v.masked)
    return v.hist ? k_persist_gl<true, false, true, false, CL>
                  : (v.block ? k_persist_gl<true, false, false, false, CL> : k_persist_gl<true, false, false, false, CL, true>);
  return v.hist ? k_persist_gl<false, false, true, false, CL>
                : (v.block ? k_persist_gl<false, false, false, false, CL> : k_persist_gl<false, false, false, false, CL, true>);
}

PlainFn pick_plain(const StepVariant& v) {
  if (v.classic) return plain_select<true>(v);
  if (v.narrow && v.vote) return v.hist ? k_plain<true, false, true, true, false, true> : k_plain<true, false, false, true, false, true>;
  if (v.narrow) return plain_select<false>(v);
  if (v.checked) return v.hist ? plain_fn<false, true, true>(v.vote) : plain_fn<false, true, false>(v.vote);
  if (v.masked) return v.hist ? plain_fn<true, false, true>(v.vote) : plain_fn<true, false, false>(v.vote);
  return v.hist ? plain_fn<false, false, true>(v.vote) : plain_fn<false, false, false>(v.vote);
}

template <bool M_, bool C_, bool H_>
StagedFn staged_fn(bool vote) {
  return vote ? k_persist<M_, C_, H_, true> : k_persist<M_, C_, H_, false>;
}

StagedFn pick_staged(const StepVariant& v) {
  // the epoch loop (generic addresses) unless checked, counting, voting or per-step
  if (!v.checked && !v.hist && !v.vote && !v.block)
    return v.masked ? k_persist<true, false, false, false, true> : k_persist<false, false, false, false, true>;
  if (v.checked) return v.hist ? staged_fn<false, true, true>(v.vote) : staged_fn<false, true, false>(v.vote);
  if (v.masked) return v.hist ? staged_fn<true, false, true>(v.vote) : staged_fn<true, false, false>(v.vote);
  return v.hist ? staged_fn<false, false, true>(v.vote) : staged_fn<false, false, false>(v.vote);
}

template <bool M_, bool C_, bool H_>
GlobalFn global_fn(bool vote) {
  return vote ? k_persist_gl<M_, C_, H_, true> : k_persist_gl<M_, C_, H_, false>;
}

GlobalFn pick_global(const StepVariant& v) {
  if (v.classic) return global_select<true>(v);
  if (v.narrow && v.vote)
    return v.hist ? k_persist_gl<true, false, true, true, false, false, true> : k_persist_gl<true, false, false, true, false, false, true>;
  if (!v.vote) return global_select<false>(v);
  if (v.checked) return v.hist ? global_fn<false, true, true>(v.vote) : global_fn<false, true, false>(v.vote);
  if (v.masked) return v.hist ? global_fn<true, false, true>(v.vote) : global_fn<true, false, false>(v.vote);
  return v.hist ? global_fn<false, false, true>(v.vote) : global_fn<false, false, false>(v.vote);
}

const void* persist_symbol(const StepVariant& v, bool staged) {
  return staged ? (const void*)pick_staged(v) : (const void*)pick_global(v);
}

}  // namespace

// 4-byte program words widened to 8 bytes with sign extension: four per
// thread per iteration (one 16-byte load, two 16-byte stores), the tail one
// by one.
__global__ void __launch_bounds__(256) k_widen(const int32_t* __restrict__ src, uint64_t* __restrict__ dst,
                                               uint64_t count) {
  const uint64_t quads = count / 4u;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < quads; q += stride) {
    const int4 w = reinterpret_cast<const int4*>(src)[q];
    reinterpret_cast<longlong2*>(dst)[2 * q] = make_longlong2(w.x, w.y);
    reinterpret_cast<longlong2*>(dst)[2 * q + 1] = make_longlong2(w.z, w.w);
  }
  for (uint64_t k = 4u * quads + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < count; k += stride)
    dst[k] = (uint64_t)(int64_t)src[k];
}

cudaError_t launch_widen(const int32_t* src, uint64_t* dst, uint64_t count, cudaStream_t stream) {
  if (!count) return cudaSuccess;
  uint64_t blocks = (count / 4u + 255u) / 256u;
  const uint64_t cap = (uint64_t)num_sms() * 16u;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  k_widen<<<(uint32_t)blocks, 256, 0, stream>>>(src, dst, count);
  return cudaGetLastError();
}

cudaError_t launch_pack(const DevState& S, const uint64_t* prog, const int32_t* prog32, const uint64_t* prog_off,
                        const uint32_t* prog_of_vm, uint32_t num_vms, uint64_t wmask, uint32_t sp,
                        bool lazy, cudaStream_t stream) {
  if (!num_vms) return cudaSuccess;
  // chunks of cl VMs per warp: 32, or fewer while that leaves under four
  // waves of chunks for the resident warps (small batches keep every SM busy)
  const uint32_t resident = (uint32_t)num_sms() * 64u;
  uint32_t cl = 32u;
  while (cl > 1u && num_vms / cl < 4u * resident) cl >>= 1;
  const uint32_t warps_needed = (num_vms + cl - 1u) / cl;
  uint32_t blocks = (warps_needed + 7u) / 8u;
  const uint32_t cap = (uint32_t)num_sms() * 64u;   // up to eight waves of resident blocks
  if (blocks > cap) blocks = cap;
  if (prog32)
    k_pack<int32_t><<<blocks, 256, 0, stream>>>(S, prog32, prog_off, prog_of_vm, num_vms, wmask, sp, lazy ? 1u : 0u,
                                                cl);
  else
    k_pack<uint64_t><<<blocks, 256, 0, stream>>>(S, prog, prog_off, prog_of_vm, num_vms, wmask, sp, lazy ? 1u : 0u,
                                                 cl);
  return cudaGetLastError();
}

using SharedFn = void (*)(DevState, Params, const uint64_t*, const uint64_t*, const uint32_t*, const uint32_t*,
                         uint32_t, uint32_t);

SharedFn pick_shared(const StepVariant& v) {
  if (v.checked) return v.hist ? k_shared<false, true, true> : k_shared<false, true, false>;
  if (v.hist) return v.masked ? k_shared<true, false, true> : k_shared<false, false, true>;
  if (v.block) return v.masked ? k_shared<true, false, false> : k_shared<false, false, false>;
  return v.masked ? k_shared_loop<true> : k_shared_loop<false>;
}

cudaError_t launch_shared(const StepVariant& var, const DevState& S, const Params& P, const uint64_t* prog,
                          const uint64_t* prog_off, const uint32_t* pv_off, const uint32_t* pv_ids,
                          uint32_t num_programs, uint32_t max_plen, uint32_t epoch, cudaStream_t stream) {
  if (!num_programs) return cudaSuccess;
  const size_t smem = (size_t)((max_plen + 1u) & ~1u) * 8u;
  SharedFn fn = pick_shared(var);
  if (smem > 48u * 1024u) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return cudaGetLastError();
  }
  uint32_t grid = num_programs;
  const uint32_t cap = (uint32_t)num_sms() * 64u;
  if (grid > cap) grid = cap;
  fn<<<grid, 128, smem, stream>>>(S, P, prog, prog_off, pv_off, pv_ids, num_programs, epoch ? epoch : 128u);
  return cudaGetLastError();
}

cudaError_t launch_materialize(const DevState& S, const uint64_t* prog, const uint64_t* prog_off,
                               const uint32_t* prog_of_vm, uint32_t num_vms, uint64_t wmask, cudaStream_t stream) {
  if (!num_vms) return cudaSuccess;
  uint32_t blocks = (num_vms + 7u) / 8u;
  const uint32_t cap = (uint32_t)num_sms() * 16u;
  if (blocks > cap) blocks = cap;
  k_materialize<<<blocks, 256, 0, stream>>>(S, prog, prog_off, prog_of_vm, num_vms, wmask);
  return cudaGetLastError();
}

void plain_configure(const StepVariant& var) {
  cudaFuncSetAttribute(pick_plain(var), cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxL1);
  cudaGetLastError();
}

cudaError_t launch_plain(const StepVariant& var, const DevState& S, const Params& P, const uint32_t* ids,
                         uint32_t count, cudaStream_t stream) {
  if (!count) return cudaSuccess;
  const uint32_t blocks = (count + 255u) / 256u;
  pick_plain(var)<<<blocks, 256, 0, stream>>>(S, P, ids, count);
  return cudaGetLastError();
}

// The variant of a persistent launch: the shape may choose the per-step form.
StepVariant shape_variant(StepVariant v, const PersistShape& sh) {
  v.block = v.block || sh.block;
  return v;
}

int persist_configure(const StepVariant& var, PersistShape& sh) {
  const void* fn = persist_symbol(shape_variant(var, sh), sh.staged);
  const size_t per_warp = sh.staged ? (32ull + 32ull * sh.slot_words) * 8ull : 0u;
  sh.smem = per_warp * sh.warps;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // staged: all of the unified L1/shared array as shared memory; otherwise
  // keep it as L1 for the M slabs in HBM
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                       sh.staged ? (int)cudaSharedmemCarveoutMaxShared : (int)cudaSharedmemCarveoutMaxL1);
  cudaGetLastError();
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)(32u * sh.warps), sh.smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  sh.grid = (uint32_t)(per_sm * num_sms());
  sh.ctas_per_sm = (uint32_t)per_sm;
  return per_sm;
}

cudaError_t launch_persist(const StepVariant& var, const DevState& S, const Params& P, const Queue& Q,
                           const PersistShape& sh, cudaStream_t stream) {
  if ((!Q.count && !Q.dcount) || !sh.grid) return cudaSuccess;
  uint32_t grid = sh.grid;
  const uint32_t warps_needed = (Q.count + 31u) / 32u;   // with dcount, Q.count is an upper bound
  const uint32_t max_useful = (warps_needed + sh.warps - 1u) / sh.warps;
  if (grid > max_useful) grid = max_useful;
  // the last (resident lanes) positions are the tail: served one VM at a
  // time to idle lanes so that no lane queues a second VM behind a running one
  Queue q = Q;
  const uint64_t lanes = (uint64_t)grid * sh.warps * 32u;
  q.soft_end = Q.count > lanes ? (uint32_t)(Q.count - lanes) : 0u;
  const StepVariant v = shape_variant(var, sh);
  if (sh.staged)
    pick_staged(v)<<<grid, 32u * sh.warps, sh.smem, stream>>>(S, P, q, sh.ncap, sh.slot_words, sh.epoch,
                                                                 sh.refill_min,
                                                                 inject_wait_expiry() ? 0u : WAIT_LIMIT);
  else
    pick_global(v)<<<grid, 32u * sh.warps, 0, stream>>>(S, P, q, sh.epoch, sh.idle_exit);
  return cudaGetLastError();
}

cudaError_t launch_tau_hist(const DevState& S, uint32_t num_vms, const uint64_t* edges, uint32_t nbins,
                            unsigned long long* counts, unsigned long long* other, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counts, 0, 8ull * nbins, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(other, 0, 8 * 4, stream);
  if (e != cudaSuccess || !num_vms) return e;
  const size_t smem = 8ull * (nbins + 1) + 4ull * nbins;
  if (smem > 48u * 1024u) {
    e = cudaFuncSetAttribute(k_tau_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  uint32_t blocks = (num_vms + 255u) / 256u;
  const uint32_t cap = (uint32_t)num_sms() * 4u;
  if (blocks > cap) blocks = cap;
  k_tau_hist<<<blocks, 256, smem, stream>>>(S.steps, S.status, num_vms, edges, nbins, counts, other);
  return cudaGetLastError();
}

cudaError_t launch_compact(const uint32_t* ids, uint32_t count, const uint8_t* status, uint32_t* out,
                           uint32_t* out_count, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(out_count, 0, sizeof(uint32_t), stream);
  if (e != cudaSuccess || !count) return e;
  uint32_t blocks = (count + 255u) / 256u;
  const uint32_t cap = (uint32_t)num_sms() * 8u;
  if (blocks > cap) blocks = cap;
  k_compact<<<blocks, 256, 0, stream>>>(ids, count, status, out, out_count);
  return cudaGetLastError();
}

cudaError_t launch_topk(const DevState& S, uint32_t num_vms, uint32_t k, TopCand* cand, TopCand* best,
                        cudaStream_t stream) {
  // at most ceil(num_vms / 1024) blocks (the candidate array is sized so)
  uint32_t blocks = (num_vms + (TOPK_TILE - k) - 1) / (TOPK_TILE - k);
  if (blocks > kMaxTopBlocks) blocks = kMaxTopBlocks;
  if (blocks == 0) blocks = 1;
  k_topk<<<blocks, 1024, 0, stream>>>(S.steps, S.status, nullptr, num_vms, k, cand);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_topk<<<1, 1024, 0, stream>>>(nullptr, nullptr, cand, blocks * k, k, best);
  return cudaGetLastError();
}

// Byte fill of device memory with 16-byte stores (p 16-byte aligned): the
// state-store resets of a batch, as a kernel of this library so that it asks
// for the same L1/shared split as the kernels that may be resident beside it.
__global__ void __launch_bounds__(256) k_fill(uint8_t* __restrict__ p, uint32_t word, uint64_t bytes) {
  const uint64_t n16 = bytes >> 4;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint4 w = make_uint4(word, word, word, word);
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n16; k += stride)
    reinterpret_cast<uint4*>(p)[k] = w;
  const uint64_t rest = bytes & 15u;
  if (blockIdx.x == 0 && threadIdx.x < rest) p[(n16 << 4) + threadIdx.x] = (uint8_t)word;
}

cudaError_t fill_bytes(void* p, uint8_t value, uint64_t bytes, cudaStream_t stream) {
  if (!bytes) return cudaSuccess;
  if (reinterpret_cast<uintptr_t>(p) & 15u) return cudaMemsetAsync(p, value, bytes, stream);
  uint64_t blocks = ((bytes >> 4) + 255u) / 256u;
  if (blocks > (uint64_t)num_sms() * 4u) blocks = (uint64_t)num_sms() * 4u;
  if (blocks == 0) blocks = 1;
  k_fill<<<(uint32_t)blocks, 256, 0, stream>>>((uint8_t*)p, 0x01010101u * value, bytes);
  return cudaGetLastError();
}

namespace {

using ServeFn = void (*)(ServeArgs, Params);

ServeFn pick_serve(const StepVariant& v) {
  if (v.checked) return k_serve<false, true, false>;
  if (v.classic) return v.masked ? k_serve<true, false, true> : k_serve<false, false, true>;
  return v.masked ? k_serve<true, false, false> : k_serve<false, false, false>;
}

}  // namespace

int serve_configure(const StepVariant& var, ServeShape& sh) {
  const ServeFn fn = pick_serve(var);
  // the kernels a request's admission launches while the serving kernel is
  // resident (state resets, pack, ring fill and publish) ask for the same L1/shared split,
  // so that an SM can host them beside it
  const void* beside[] = {(const void*)fn, (const void*)k_pack<uint64_t>, (const void*)k_pack<int32_t>,
                          (const void*)k_ring_fill, (const void*)k_ring_publish, (const void*)k_fill};
  for (const void* f : beside)
    cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxL1);
  cudaGetLastError();
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 128, 0) != cudaSuccess || per_sm <= 0) {
    cudaGetLastError();
    return 0;
  }
  sh.threads = 128;
  sh.grid = (uint32_t)(per_sm > 1 ? per_sm - 1 : 1) * (uint32_t)num_sms();
  return per_sm;
}

cudaError_t launch_serve(const StepVariant& var, const ServeArgs& A, const Params& P, const ServeShape& sh,
                         cudaStream_t stream) {
  pick_serve(var)<<<sh.grid, sh.threads, 0, stream>>>(A, P);
  return cudaGetLastError();
}

cudaError_t launch_ring_append(uint64_t* ring, uint64_t mask, unsigned long long start, uint32_t slot,
                               const uint32_t* ids, uint32_t count, unsigned long long* credits,
                               cudaStream_t stream) {
  if (count) {
    uint32_t blocks = (count + 255u) / 256u;
    if (blocks > (uint32_t)num_sms() * 4u) blocks = (uint32_t)num_sms() * 4u;
    k_ring_fill<<<blocks, 256, 0, stream>>>(ring, mask, start, slot, ids, count);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_ring_publish<<<1, 1, 0, stream>>>(credits, count);
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
