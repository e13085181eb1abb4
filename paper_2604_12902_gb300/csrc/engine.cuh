// engine.cuh -- device-side word-RASP step for sm_103a.
//
// One call of `one_step` applies the Sec. 2.1 transition of "Towards a
// Linear-Algebraic Hypervisor" to one machine held in registers (i, a, u_0,
// y_0, steps) plus its memory M, tape u_1..u_l and output y_1..y_s (in shared
// memory or HBM, whichever the schedule chose). The case equation is
// evaluated in its guarded-sum form (Sec. 2.1, Phi_w(c) = sum_psi
// eta_psi(c) Phi_psi(c), exactly one guard true): every candidate update is
// formed and the guards select, so a warp whose lanes hold different opcodes
// executes one instruction stream.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rasp {

enum : uint32_t {
  ST_RUNNING = 0, ST_HALTED = 1, ST_TIMEOUT = 2, ST_FAULT_OVERFLOW = 3, ST_FAULT_ADDR = 4,
  CONT = 0xFFu  // step applied, machine continues
};

enum : int { ERR_NONE = 0, ERR_WAIT_TIMEOUT = 1 };

// Structure-of-arrays state store in HBM (one entry per VM).
struct DevState {
  uint64_t* i;
  uint64_t* a;
  uint64_t* steps;
  const uint64_t* cap;
  uint8_t* status;
  uint32_t* uhead;            // u_0
  uint32_t* ylen;             // y_0
  const uint32_t* n;          // memory words
  const uint64_t* mem_off;    // word offset of the VM's M slab (even)
  uint64_t* mem;              // M slabs
  const uint64_t* tape;       // u_1..u_l, stride ellp words per VM
  uint64_t* y;                // y_1..y_s, stride sp words per VM
};

struct Params {
  uint64_t wmask;             // 2^w - 1
  uint64_t budget;            // max_steps of this rasp_run
  uint32_t ell, s;            // l, s
  uint32_t ellp, sp;          // padded strides (even)
  int* err;                   // internal error flag (bounded waits)
  unsigned long long* hist;   // [10]: 1..7 per opcode, 8 PRI-full, 9 BNZ-taken
};

struct Queue {
  const uint32_t* ids;        // VM ids in schedule order
  uint32_t count;
  uint32_t* head;             // next unclaimed position (reset to 0 per launch)
};

// Registers of one machine while it runs.
struct Regs {
  uint64_t i, a, steps, stop, cap;
  uint32_t ip;                // i mod n
  uint32_t n;
  uint32_t u0, y0;
};

struct Hist {
  uint32_t c[10];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 10; ++k) c[k] = 0;
  }
};

__device__ __forceinline__ uint32_t mod_n(uint64_t x, uint32_t n) {
  // x mod n on the unsigned value (words are bit vectors, Sec. 2.1).
  if (x < n) return (uint32_t)x;
  if ((n & (n - 1)) == 0) return (uint32_t)(x & (n - 1));
  return (uint32_t)(x % n);
}

// One transition (or the decision that none applies).
// Returns CONT after applying a step, otherwise the machine's final status
// for this run: HALTED (fixed point), a CHECKED fault, or, when
// steps >= stop, TIMEOUT (steps >= cap) / RUNNING (budget reached).
template <bool MASKED, bool CHECKED, bool HIST>
__device__ __forceinline__ uint32_t one_step(uint64_t* __restrict__ M,
                                             const uint64_t* __restrict__ T,
                                             uint64_t* __restrict__ Y,
                                             const Params& P, Regs& r, Hist& h) {
  const uint64_t wm = MASKED ? P.wmask : ~0ull;
  const uint64_t i = r.i, a = r.a;
  const uint32_t ip = r.ip, n = r.n;
  if (CHECKED) {
    // without circular addressing the fetch needs i, i+1 in [0, n)
    if (!(i < (uint64_t)n - 1)) {
      if (r.steps >= r.stop) return r.steps >= r.cap ? ST_TIMEOUT : ST_RUNNING;
      return ST_FAULT_ADDR;
    }
  }
  // fetch <o, j> = <M[i mod n], M[(i (+) 1) mod n]>
  uint64_t o, j;
  if (!(ip & 1u) && ip + 1u < n && i != wm) {
    const ulonglong2 oj = *reinterpret_cast<const ulonglong2*>(M + ip);
    o = oj.x;
    j = oj.y;
  } else {
    o = M[ip];
    uint32_t k1 = (i == wm) ? 0u : ip + 1u;   // i (+) 1 wraps to 0 at i = 2^w - 1
    if (k1 == n) k1 = 0u;
    j = M[k1];
  }
  const uint32_t jm = mod_n(j, n);
  const bool valid = (o - 1ull) < 7ull;
  const uint32_t op = valid ? (uint32_t)o : 0u;
  // guards of the "otherwise" case: c -> c
  const bool fixed = !valid || (op == 6u && r.u0 >= P.ell) || (op == 5u && a != 0 && j == i);
  if (fixed) return ST_HALTED;
  if (r.steps >= r.stop) return r.steps >= r.cap ? ST_TIMEOUT : ST_RUNNING;
  if (CHECKED) {
    if (op != 1u && op != 5u && j >= (uint64_t)n) return ST_FAULT_ADDR;
  }
  uint64_t v = 0;
  if (op == 2u || op == 3u || op == 7u) v = M[jm];
  const uint64_t sum = a + v;
  const uint64_t prod = a * v;
  if (CHECKED) {
    if (op == 2u && (int64_t)((a ^ sum) & (v ^ sum)) < 0) return ST_FAULT_OVERFLOW;
    if (op == 3u) {
      const int64_t hi = __mul64hi((long long)a, (long long)v);
      if (hi != ((int64_t)prod >> 63)) return ST_FAULT_OVERFLOW;
    }
  }
  uint64_t na = a;
  na = (op == 1u) ? j : na;
  na = (op == 2u) ? sum : na;
  na = (op == 3u) ? prod : na;
  if (MASKED) na &= wm;
  // M_{j mod n} <- a (STO) or <- u-bullet (RD); u-triangle advances the head
  if (op == 4u) M[jm] = a;
  if (op == 6u) {
    M[jm] = T[r.u0];
    r.u0 += 1u;
  }
  // y :: M_{j mod n}
  const bool put = (op == 7u) && (r.y0 < P.s);
  if (put) {
    Y[r.y0] = v;
    r.y0 += 1u;
  }
  const bool taken = (op == 5u) && (a != 0);
  if (taken) {
    r.i = j;
    r.ip = jm;
  } else {
    const uint64_t ni = (i + 2ull) & wm;
    uint32_t nip = ip + 2u;
    if (nip >= n) nip -= n;
    if (nip >= n) nip -= n;
    if (ni < i) nip = (ni < n) ? (uint32_t)ni : 0u;   // i (+) 2 wrapped past 2^w
    r.i = ni;
    r.ip = nip;
  }
  r.a = na;
  r.steps += 1ull;
  if (HIST) {
#pragma unroll
    for (uint32_t k = 1; k <= 7; ++k) h.c[k] += (op == k) ? 1u : 0u;
    h.c[8] += (op == 7u && !put) ? 1u : 0u;
    h.c[9] += taken ? 1u : 0u;
  }
  return CONT;
}

template <bool HIST>
__device__ __forceinline__ void flush_hist(const Params& P, Hist& h) {
  if constexpr (HIST) {
#pragma unroll
    for (int k = 1; k < 10; ++k) {
      unsigned long long v = h.c[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if ((threadIdx.x & 31) == 0 && v) atomicAdd(&P.hist[k], v);
    }
    h.zero();
  }
}

// Load the registers of VM v from the state store.
__device__ __forceinline__ void load_regs(const DevState& S, const Params& P, uint32_t v, Regs& r) {
  r.i = S.i[v];
  r.a = S.a[v];
  r.steps = S.steps[v];
  r.cap = S.cap[v];
  r.n = S.n[v];
  r.u0 = S.uhead[v];
  r.y0 = S.ylen[v];
  r.stop = P.budget < r.cap ? P.budget : r.cap;
  r.ip = mod_n(r.i, r.n);
}

__device__ __forceinline__ void store_regs(const DevState& S, uint32_t v, const Regs& r, uint32_t st) {
  S.i[v] = r.i;
  S.a[v] = r.a;
  S.steps[v] = r.steps;
  S.uhead[v] = r.u0;
  S.ylen[v] = r.y0;
  S.status[v] = (uint8_t)st;
}

}  // namespace rasp
