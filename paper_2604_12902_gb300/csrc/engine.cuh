// engine.cuh -- device-side word-RASP step for sm_103a.
//
// One call of `one_step` applies the Sec. 2.1 transition of "Towards a
// Linear-Algebraic Hypervisor" to one machine held in registers (i, a, u_0,
// y_0, a step countdown) plus its memory M, tape u_1..u_l and output
// y_1..y_s (in shared memory or HBM, whichever the schedule chose). The case
// equation is evaluated in its guarded-sum form (Sec. 2.1, Phi_w(c) =
// sum_psi eta_psi(c) Phi_psi(c), exactly one guard true): the candidate
// updates of LOD/ADD/MUL/STO/BNZ are formed and the guards select, so a warp
// whose lanes hold different opcodes runs one instruction stream. RD and PRI
// (a few steps per program), fetches that straddle the end of memory,
// operands outside [0, n) and the wrap of i at 2^w take short side paths.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace rasp {

enum : uint32_t {
  ST_RUNNING = 0, ST_HALTED = 1, ST_TIMEOUT = 2, ST_FAULT_OVERFLOW = 3, ST_FAULT_ADDR = 4,
  CONT = 0xFFu  // step applied, machine continues
};

enum : int { ERR_NONE = 0, ERR_WAIT_TIMEOUT = 1, ERR_SLOT = 2, ERR_RING = 3 };

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
  uint64_t* mem;              // M slabs (8-byte words)
  uint32_t* mem32;            // M slabs of a narrow batch (w <= 32: 4-byte words; NULL otherwise)
  const uint64_t* tape;       // u_1..u_l, stride ellp words per VM
  uint64_t* y;                // y_1..y_s, stride sp words per VM
  uint8_t* codedirty;         // 1 if the VM may have written into its program words (NULL: untracked)
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
  uint32_t count;             // number of ids (when dcount is NULL)
  uint32_t* head;             // next unclaimed position (reset to 0 per launch)
  uint32_t* tail_head;        // next unclaimed tail position (reset to 0 per launch)
  uint32_t soft_end;          // positions >= soft_end are handed out one by one to idle lanes
  const uint32_t* dcount;     // persistent HBM-slab kernel: if set, the number of ids is read
                              // here at launch (written by an earlier kernel on the stream) and
                              // soft_end is derived from it
};

// Registers of one machine while it runs. The instruction counter is kept
// as i = ibase + ip with ip = i mod n; ibase is 0 while i < n, which is
// where programs spend their time, so the common step touches only the
// 32-bit ip. Steps are counted down in 32 bits: the machine has taken
// steps + (left0 - left) steps; the 64-bit budget and cap are consulted only
// when the countdown reaches zero.
struct Regs {
  uint64_t a;
  uint64_t ibase;             // i - (i mod n)
  uint64_t steps;             // steps at the start of the current countdown
  uint64_t cap;               // step cap; the run stops at min(budget, cap)
  uint32_t left0, left;       // countdown start and remaining
  uint32_t ip;                // i mod n
  uint32_t n;
  uint32_t ilim;              // min(n, 2^w): while ibase = 0, ip + 2 < ilim means i (+) 2 = ip + 2 < n
  uint32_t u0, y0;
  ulonglong2 cur;             // <M[ip], M[ip+1]> when `have`: the next instruction, already loaded
  bool have;
  bool clean;                 // shared-program mode: no write has touched M[0, plen) yet
};

__device__ __forceinline__ uint64_t i_of(const Regs& r) { return r.ibase + (uint64_t)r.ip; }
__device__ __forceinline__ uint64_t steps_of(const Regs& r) { return r.steps + (uint64_t)(r.left0 - r.left); }

struct Hist {
  uint32_t c[10];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 10; ++k) c[k] = 0;
  }
};

static __device__ __noinline__ uint32_t mod_n_slow(uint64_t x, uint32_t n) {
  if ((n & (n - 1u)) == 0u) return (uint32_t)(x & (uint64_t)(n - 1u));
  return (uint32_t)(x % n);
}

// x mod n on the unsigned value (words are bit vectors, Sec. 2.1).
__device__ __forceinline__ uint32_t mod_n(uint64_t x, uint32_t n) {
  return (x < (uint64_t)n) ? (uint32_t)x : mod_n_slow(x, n);
}

// Opcode 5's condition: BNZ (word machine, Sec. 2.1) jumps when a != 0; BPA
// (classic opcode set, Sec. 1.1) when a > 0, with the w-bit word a read as a
// two's complement integer: 1 <= a <= 2^(w-1) - 1 = wm >> 1.
template <bool CLASSIC>
__device__ __forceinline__ bool jumps(uint64_t a, uint64_t wm) {
  if constexpr (CLASSIC) return (a - 1ull) < (wm >> 1);
  else return a != 0ull;
}

__device__ __forceinline__ uint64_t stop_of(const Params& P, const Regs& r) {
  return P.budget < r.cap ? P.budget : r.cap;
}

// Start a fresh 32-bit countdown toward the stop; false if already there.
__device__ __forceinline__ bool arm_countdown(const Params& P, Regs& r) {
  const uint64_t stop = stop_of(P, r);
  if (r.steps >= stop) {
    r.left0 = r.left = 0;
    return false;
  }
  const uint64_t rem = stop - r.steps;
  r.left0 = r.left = rem > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)rem;
  return true;
}

struct Countdown {
  uint64_t steps;
  uint32_t left;
  uint32_t status;   // CONT: re-armed; else TIMEOUT / RUNNING at the stop
};

// The countdown reached zero (left == 0) and the machine is not a fixed
// point: either the stop is reached or a new countdown starts.
static __device__ __noinline__ Countdown countdown_next(uint64_t steps, uint32_t left0, uint64_t stop, uint64_t cap) {
  Countdown c;
  c.steps = steps + left0;
  if (c.steps >= stop) {
    c.left = 0;
    c.status = c.steps >= cap ? ST_TIMEOUT : ST_RUNNING;
    return c;
  }
  const uint64_t rem = stop - c.steps;
  c.left = rem > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)rem;
  c.status = CONT;
  return c;
}

__device__ __forceinline__ uint32_t on_countdown_zero(const Params& P, Regs& r) {
  const Countdown c = countdown_next(r.steps, r.left0, stop_of(P, r), r.cap);
  r.steps = c.steps;
  r.left0 = r.left = c.left;
  return c.status;
}

// Result of fetching and decoding the next transition.
struct Decoded {
  uint64_t j;
  uint32_t op;      // 1..7, 0 for an invalid opcode
  uint32_t jm;      // j mod n
  bool jin;         // j < n
  bool taken;       // BNZ with a != 0
};

// ---- views of a VM's memory M
// The steps reach M through three accessors overloaded on the view. The
// plain view is a pointer to the VM's slab in HBM. ShView is the view of a
// VM whose program is shared by many VMs (Sec. 2.1's stored program, held
// once per program): words [0, plen) are served from the program's copy in
// shared memory while the VM has not written into them (Regs::clean), so a
// slab need not hold its program words at all (lazy pack). The VM's first
// write into a program word copies the program into its slab before it is
// applied (copy-on-write; harmless when the slab already holds it), after
// which every word comes from the slab. `clean` is Regs::clean; the plain
// view ignores it.
struct ShView {
  uint64_t* M;            // the VM's slab (n words)
  const uint64_t* Pg;     // the program in shared memory (plen words, masked to w)
  uint32_t plen;          // program words (even)
};

__device__ __forceinline__ ulonglong2 mem_pair(const uint64_t* M, bool, uint32_t k) {
  return *reinterpret_cast<const ulonglong2*>(M + k);
}
__device__ __forceinline__ uint64_t mem_rd(const uint64_t* M, bool, uint32_t k) { return M[k]; }
__device__ __forceinline__ void mem_wr(uint64_t* M, bool&, uint32_t k, uint64_t v) { M[k] = v; }

// k even; plen is even, so the pair lies wholly inside or outside [0, plen)
__device__ __forceinline__ ulonglong2 mem_pair(const ShView& V, bool clean, uint32_t k) {
  const uint64_t* src = (clean && k < V.plen) ? V.Pg : V.M;
  return *reinterpret_cast<const ulonglong2*>(src + k);
}
__device__ __forceinline__ uint64_t mem_rd(const ShView& V, bool clean, uint32_t k) {
  return (clean && k < V.plen) ? V.Pg[k] : V.M[k];
}
// The program into the VM's own slab (the VM's first write into a program
// word).
static __device__ __noinline__ void sh_copy_program(uint64_t* M, const uint64_t* Pg, uint32_t plen) {
  for (uint32_t k = 0; k < plen; k += 2u)
    *reinterpret_cast<ulonglong2*>(M + k) = *reinterpret_cast<const ulonglong2*>(Pg + k);
}
__device__ __forceinline__ void mem_wr(const ShView& V, bool& clean, uint32_t k, uint64_t v) {
  if (clean && k < V.plen) {
    sh_copy_program(V.M, V.Pg, V.plen);
    clean = false;
  }
  V.M[k] = v;
}

// The view of a VM of a narrow batch (w <= 32): M holds 4-byte words, the
// same values as 8-byte words would (every word is below 2^w). Pairs are
// 8-byte aligned (k even, slabs start at an even word).
struct NarrowView {
  uint32_t* M;
};
__device__ __forceinline__ ulonglong2 mem_pair(const NarrowView& V, bool, uint32_t k) {
  const uint2 p = *reinterpret_cast<const uint2*>(V.M + k);
  return make_ulonglong2(p.x, p.y);
}
__device__ __forceinline__ uint64_t mem_rd(const NarrowView& V, bool, uint32_t k) { return V.M[k]; }
__device__ __forceinline__ void mem_wr(const NarrowView& V, bool&, uint32_t k, uint64_t v) { V.M[k] = (uint32_t)v; }

// A lane's memory in shared memory (the SMEM-staged schedule): the plain
// accessors through a generic pointer; its epoch loop addresses M, the tape
// and y generically.
struct SmemView {
  uint64_t* M;
};
__device__ __forceinline__ ulonglong2 mem_pair(const SmemView& V, bool, uint32_t k) {
  return *reinterpret_cast<const ulonglong2*>(V.M + k);
}
__device__ __forceinline__ uint64_t mem_rd(const SmemView& V, bool, uint32_t k) { return V.M[k]; }
__device__ __forceinline__ void mem_wr(const SmemView& V, bool&, uint32_t k, uint64_t v) { V.M[k] = v; }

// <o, j> = <M[i mod n], M[(i (+) 1) mod n]> when the pair is not one aligned
// 16-byte word (odd n or odd i mod n, or i = 2^w - 1 where i (+) 1 wraps to 0).
template <class Mem>
__device__ __noinline__ ulonglong2 fetch_slow(Mem M, bool clean, uint32_t ip, uint32_t n, uint64_t i, uint64_t wm) {
  if (!(ip & 1u) && ip + 1u < n && i != wm) return mem_pair(M, clean, ip);
  ulonglong2 oj;
  oj.x = mem_rd(M, clean, ip);
  uint32_t k1 = (i == wm) ? 0u : ip + 1u;
  if (k1 == n) k1 = 0u;
  oj.y = mem_rd(M, clean, k1);
  return oj;
}

// Fetch, decode and evaluate the guards of the next transition. Returns CONT
// if the transition applies (d filled), else the machine's final status for
// this run: HALTED (fixed point), a CHECKED fault, or TIMEOUT / RUNNING at
// the step stop.
template <bool MASKED, bool CHECKED, bool CLASSIC = false, class Mem>
__device__ __forceinline__ uint32_t decode(Mem M, const Params& P, Regs& r, Decoded& d) {
  const uint64_t wm = MASKED ? P.wmask : ~0ull;
  const uint32_t ip = r.ip, n = r.n;
  const bool wide = r.ibase != 0ull;      // i >= n
  if constexpr (CHECKED) {
    // without circular addressing the fetch needs i, i+1 in [0, n)
    if (wide | (ip + 1u >= n)) {
      if (r.left == 0u) {
        const uint32_t s = on_countdown_zero(P, r);
        if (s != CONT) return s;
      }
      return ST_FAULT_ADDR;
    }
  }
  ulonglong2 oj;
  if (((ip | n) & 1u) == 0u) {
    // even n and even i mod n: i is even (ibase is a multiple of n), so
    // i != 2^w - 1 and M[ip], M[ip+1] is one aligned 16-byte word
    oj = mem_pair(M, r.clean, ip);
  } else {
    oj = fetch_slow(M, r.clean, ip, n, i_of(r), wm);
  }
  const uint64_t o = oj.x, j = oj.y;
  d.j = j;
  d.jin = j < (uint64_t)n;
  d.op = ((o - 1ull) < 7ull) ? (uint32_t)o : 0u;
  d.taken = (d.op == 5u) & jumps<CLASSIC>(r.a, wm);
  // j mod n only where j is an address or a jump target (LOD's j is an
  // immediate, an untaken BNZ ignores it)
  const bool addr = ((d.op >= 2u) & (d.op != 5u)) | d.taken;
  d.jm = (d.jin | !addr) ? (uint32_t)j : mod_n_slow(j, n);
  // guards of the "otherwise" case (c -> c): invalid opcode, RD at the end
  // of the tape, BNZ to itself (j == i; while i < n that is j < n and
  // j == i mod n)
  bool fixed = (d.op == 0u) | ((d.op == 6u) & (r.u0 >= P.ell)) | (d.taken & d.jin & ((uint32_t)j == ip) & !wide);
  if (wide && d.taken && j == i_of(r)) fixed = true;
  if (fixed | (r.left == 0u)) {
    if (fixed) return ST_HALTED;
    const uint32_t s = on_countdown_zero(P, r);
    if (s != CONT) return s;
  }
  if constexpr (CHECKED) {
    if ((d.op != 1u) & (d.op != 5u) & !d.jin) return ST_FAULT_ADDR;
  }
  return CONT;
}

// i <- j (taken BNZ) or i (+) 2, kept as ibase + ip.
template <bool MASKED>
__device__ __forceinline__ void advance(const Params& P, Regs& r, const Decoded& d) {
  if (d.taken) {
    r.ip = d.jm;
    r.ibase = d.jin ? 0ull : d.j - d.jm;
  } else {
    uint32_t nip = r.ip + 2u;
    if ((r.ibase != 0ull) | (nip >= r.ilim)) {
      // end of memory, i >= n, or i (+) 2 wraps at 2^w
      const uint64_t wm = MASKED ? P.wmask : ~0ull;
      const uint64_t ni = (i_of(r) + 2ull) & wm;
      nip = mod_n(ni, r.n);
      r.ibase = ni - nip;
    }
    r.ip = nip;
  }
  r.left -= 1u;
}

template <bool HIST>
__device__ __forceinline__ void count_step(Hist& h, uint32_t op, bool taken) {
  if constexpr (HIST) {
#pragma unroll
    for (uint32_t k = 1; k <= 7; ++k) h.c[k] += (op == k) ? 1u : 0u;
    h.c[9] += taken ? 1u : 0u;
  }
}

// One transition, general form: every case of the Sec. 2.1 equation,
// every guard and every wrap. Returns CONT after applying it, else the final
// status (see decode).
template <bool MASKED, bool CHECKED, bool HIST, bool CLASSIC = false, class Mem>
__device__ __forceinline__ uint32_t step_general(Mem M, const uint64_t* __restrict__ T, uint64_t* __restrict__ Y,
                                                 const Params& P, Regs& r, Hist& h) {
  Decoded d;
  const uint32_t s = decode<MASKED, CHECKED, CLASSIC>(M, P, r, d);
  if (s != CONT) return s;
  const uint32_t op = d.op, jm = d.jm;
  const uint64_t a = r.a;
  uint64_t v = 0;
  if ((op == 2u) | (op == 3u)) v = mem_rd(M, r.clean, jm);
  const uint64_t sum = a + v;
  const uint64_t prod = CLASSIC ? a - v : a * v;    // opcode 3: MUL, or SUB in the classic set
  if constexpr (CHECKED) {
    if ((op == 2u) & ((int64_t)((a ^ sum) & (v ^ sum)) < 0)) return ST_FAULT_OVERFLOW;
    if constexpr (CLASSIC) {
      if ((op == 3u) & ((int64_t)((a ^ v) & (a ^ prod)) < 0)) return ST_FAULT_OVERFLOW;
    } else {
      if ((op == 3u) && __mul64hi((long long)a, (long long)v) != ((int64_t)prod >> 63)) return ST_FAULT_OVERFLOW;
    }
  }
  uint64_t na = (op == 1u) ? d.j : a;
  na = (op == 2u) ? sum : na;
  na = (op == 3u) ? prod : na;
  if (MASKED) na &= P.wmask;
  if (op == 4u) mem_wr(M, r.clean, jm, a);       // M_{j mod n} <- a
  if (op >= 6u) {
    if (op == 6u) {                              // M_{j mod n} <- u-bullet; u-triangle
      mem_wr(M, r.clean, jm, T[r.u0]);
      r.u0 += 1u;
    } else {                                     // y :: M_{j mod n}
      const uint64_t pv = mem_rd(M, r.clean, jm);
      if (r.y0 < P.s) {
        Y[r.y0] = pv;
        r.y0 += 1u;
      } else if (HIST) {
        h.c[8] += 1u;
      }
    }
  }
  r.a = na;
  advance<MASKED>(P, r, d);
  count_step<HIST>(h, op, d.taken);
  return CONT;
}

// One transition in guarded-sum form. The common case -- i < n with an
// aligned instruction pair, a valid opcode whose operand j lies in [0, n),
// no fixed point, no wrap, countdown not exhausted -- is evaluated without
// branches: every candidate update is formed and the opcode guards select
// (Phi_w(c) = sum_psi eta_psi(c) Phi_psi(c)), so lanes holding different
// opcodes stay on one instruction stream. Anything else falls through to
// step_general.
//
// With PIPE the fast path is software-pipelined: the instruction pair
// <o, j> of the current step was loaded by the previous step (r.cur), and at
// the start of this step two independent 16-byte loads go out together --
// the sequential next pair M[ip+2..ip+3] and the aligned pair holding
// M[j mod n], which is both the operand of ADD/MUL/PRI and the first
// instruction of a taken BNZ. A step then waits on one memory latency
// instead of two in a row, at the price of more registers and loads. A
// STO/RD that writes the prefetched pair invalidates it.

// Load the instruction pair at i into r.cur when the fast path can use it:
// r.have is true iff i < n, i is even and i + 1 < n (i even and 2^w - 1 odd,
// so i (+) 1 = i + 1), and then r.cur = <M[i], M[i+1]>.
template <class Mem>
__device__ __forceinline__ void prime(Mem M, Regs& r) {
  r.have = (r.ibase == 0ull) & ((r.ip & 1u) == 0u) & (r.ip + 1u < r.n);
  if (r.have) r.cur = mem_pair(M, r.clean, r.ip);
}

// Fast path of the default step (WRAP, no counters; any w) as one
// predicated PTX block, the same guarded-sum evaluation as the C++ fast path
// of one_step below but without a branch: the two pair loads (sequential
// next pair, aligned pair holding M[j mod n]) go out together, every guard is
// a predicate, and every update -- a, M[j mod n], y, u_0, y_0, i, the next
// pair and its flag -- is committed under the predicate "not rare". Rare: an
// invalid opcode, an operand outside [0, n), the end of the countdown, RD at
// the end of the tape, BNZ to itself, i (+) 2 reaching n or 2^w, a store into the
// pair just loaded for the next step (self-modifying code). Precondition
// (have): i = ip < n, ip even, ip + 1 < n, <co, cj> = <M[ip], M[ip+1]>.
// Returns 1, and changes nothing, when the step needs the general path.
#define RASP_FAST_STEP_A1 \
      "{\n\t" \
      ".reg .pred pv, pj, pz, pt, pq, prd, pl, po, pa, px, pk, p1, p2, p3, p6, p7, pw, pp, ph, pg;\n\t" \
      ".reg .b32 op, oh, jm, jh, t0, t1, t2, nip, ip3;\n\t" \
      ".reg .b64 sx, sy, qx, qy, v, sm, pd, na, w, ad, am;\n\t" \
      "mov.b64 {op, oh}, %1;\n\t" \
      "mov.b64 {jm, jh}, %2;\n\t" \
      "add.u32 t0, op, -1;\n\t" \
      "setp.lt.u32 pv, t0, 7;\n\t" \
      "setp.eq.and.u32 pv, oh, 0, pv;\n\t" \
      "setp.lt.u32 pj, jm, %12;\n\t" \
      "setp.eq.and.u32 pj, jh, 0, pj;\n\t"
#define RASP_FAST_STEP_A2 \
      "setp.eq.and.u32 pt, op, 5, pz;\n\t" \
      "add.u32 ip3, %3, 3;\n\t" \
      "setp.lt.u32 pq, ip3, %12;\n\t" \
      "mad.wide.u32 ad, %3, 8, %9;\n\t" \
      "@pq ld.global.v2.u64 {sx, sy}, [ad+16];\n\t" \
      "mov.b32 t1, 0x8C;\n\t" \
      "shr.b32 t1, t1, op;\n\t" \
      "and.b32 t1, t1, 1;\n\t" \
      "setp.ne.or.u32 prd, t1, 0, pt;\n\t" \
      "and.pred pl, prd, pj;\n\t" \
      "and.b32 t0, jm, -2;\n\t" \
      "mad.wide.u32 ad, t0, 8, %9;\n\t" \
      "@pl ld.global.v2.u64 {qx, qy}, [ad];\n\t" \
      "and.b32 t2, jm, 1;\n\t" \
      "setp.ne.u32 po, t2, 0;\n\t" \
      "selp.b64 v, qy, qx, po;\n\t" \
      "add.u64 sm, %0, v;\n\t"
#define RASP_FAST_STEP_A3 \
      "mov.b32 t1, 0xDC;\n\t" \
      "shr.b32 t1, t1, op;\n\t" \
      "and.b32 t1, t1, 1;\n\t" \
      "setp.ne.or.u32 pa, t1, 0, pt;\n\t" \
      "setp.eq.u32 p6, op, 6;\n\t" \
      "setp.eq.or.u32 pw, op, 4, p6;\n\t" \
      "setp.ge.and.u32 px, %6, %13, p6;\n\t" \
      "setp.eq.or.u32 px, %5, 0, px;\n\t" \
      "not.pred ph, pj;\n\t" \
      "and.pred ph, ph, pa;\n\t" \
      "or.pred px, px, ph;\n\t" \
      "not.pred ph, pv;\n\t" \
      "or.pred px, px, ph;\n\t" \
      "setp.eq.and.u32 ph, jm, %3, pt;\n\t" \
      "or.pred px, px, ph;\n\t" \
      "add.u32 nip, %3, 2;\n\t" \
      "setp.ge.and.u32 ph, nip, %15, !pt;\n\t" \
      "or.pred px, px, ph;\n\t" \
      "or.b32 t0, jm, 1;\n\t" \
      "setp.eq.and.u32 ph, t0, ip3, pw;\n\t" \
      "or.pred px, px, ph;\n\t" \
      "not.pred pk, px;\n\t" \
      "setp.eq.u32 p1, op, 1;\n\t" \
      "setp.eq.u32 p2, op, 2;\n\t" \
      "setp.eq.u32 p3, op, 3;\n\t" \
      "selp.b64 na, %2, %0, p1;\n\t" \
      "selp.b64 na, sm, na, p2;\n\t" \
      "selp.b64 na, pd, na, p3;\n\t" \
      "and.pred pw, pw, pk;\n\t" \
      "and.pred pg, p6, pk;\n\t" \
      "mov.b64 w, %0;\n\t" \
      "mad.wide.u32 ad, %6, 8, %10;\n\t" \
      "@pg ld.global.u64 w, [ad];\n\t" \
      "mad.wide.u32 ad, jm, 8, %9;\n\t" \
      "@pw st.global.u64 [ad], w;\n\t" \
      "setp.eq.u32 p7, op, 7;\n\t" \
      "setp.lt.and.u32 pp, %7, %14, p7;\n\t" \
      "and.pred pp, pp, pk;\n\t" \
      "mad.wide.u32 ad, %7, 8, %11;\n\t" \
      "@pp st.global.u64 [ad], v;\n\t" \
      "@pg add.u32 %6, %6, 1;\n\t" \
      "@pp add.u32 %7, %7, 1;\n\t"
// opcode 5's condition (pz) and opcode 3's result (pd): word machine BNZ and
// MUL; classic set BPA (1 <= a <= 2^(w-1) - 1, %17 = 2^(w-1) - 1) and SUB
#define RASP_FAST_STEP_PZ_WORD "setp.ne.u64 pz, %0, 0;\n\t"
#define RASP_FAST_STEP_PD_WORD "mul.lo.u64 pd, %0, v;\n\t"
#define RASP_FAST_STEP_PZ_CLASSIC "add.u64 am, %0, -1;\n\tsetp.lt.u64 pz, am, %17;\n\t"
#define RASP_FAST_STEP_PD_CLASSIC "sub.u64 pd, %0, v;\n\t"
#define RASP_FAST_STEP_B \
      "@pk mov.b64 %0, na;\n\t" \
      "@pk selp.b64 %1, qx, sx, pt;\n\t" \
      "@pk selp.b64 %2, qy, sy, pt;\n\t" \
      "add.u32 t1, jm, 1;\n\t" \
      "setp.lt.u32 p3, t1, %12;\n\t" \
      "setp.eq.and.u32 p3, t2, 0, p3;\n\t" \
      "selp.u32 t1, 1, 0, p3;\n\t" \
      "selp.u32 t0, 1, 0, pq;\n\t" \
      "@pk selp.u32 %8, t1, t0, pt;\n\t" \
      "@pk selp.b32 %3, jm, nip, pt;\n\t" \
      "@pk sub.u32 %5, %5, 1;\n\t" \
      "selp.u32 %4, 1, 0, px;\n\t" \
      "}"
#define RASP_FAST_STEP_OPERANDS                                                                   \
  : "+l"(a), "+l"(co), "+l"(cj), "+r"(ip), "=r"(rare), "+r"(left), "+r"(u0), "+r"(y0), "+r"(have) \
  : "l"(M), "l"(T), "l"(Y), "r"(n), "r"(ell), "r"(s), "r"(ilim), "l"(wmask), "l"(wmask >> 1)     \
  : "memory"

template <bool MASKED, bool CLASSIC>
__device__ __forceinline__ uint32_t fast_step_ptx(uint64_t* M, const uint64_t* T, uint64_t* Y, uint32_t n,
                                                  uint32_t ell, uint32_t s, uint64_t& a, uint64_t& co,
                                                  uint64_t& cj, uint32_t& ip, uint32_t& left, uint32_t& u0,
                                                  uint32_t& y0, uint32_t& have, uint32_t ilim, uint64_t wmask) {
  uint32_t rare;
  // w < 64: the new accumulator is reduced to w bits (%16 = 2^w - 1); i (+) 2
  // must stay below ilim = min(n, 2^w)
  if constexpr (MASKED && CLASSIC) {
    asm volatile(RASP_FAST_STEP_A1 RASP_FAST_STEP_PZ_CLASSIC RASP_FAST_STEP_A2 RASP_FAST_STEP_PD_CLASSIC
                 RASP_FAST_STEP_A3 "and.b64 na, na, %16;\n\t" RASP_FAST_STEP_B RASP_FAST_STEP_OPERANDS);
  } else if constexpr (MASKED) {
    asm volatile(RASP_FAST_STEP_A1 RASP_FAST_STEP_PZ_WORD RASP_FAST_STEP_A2 RASP_FAST_STEP_PD_WORD
                 RASP_FAST_STEP_A3 "and.b64 na, na, %16;\n\t" RASP_FAST_STEP_B RASP_FAST_STEP_OPERANDS);
  } else if constexpr (CLASSIC) {
    asm volatile(RASP_FAST_STEP_A1 RASP_FAST_STEP_PZ_CLASSIC RASP_FAST_STEP_A2 RASP_FAST_STEP_PD_CLASSIC
                 RASP_FAST_STEP_A3 RASP_FAST_STEP_B RASP_FAST_STEP_OPERANDS);
  } else {
    asm volatile(RASP_FAST_STEP_A1 RASP_FAST_STEP_PZ_WORD RASP_FAST_STEP_A2 RASP_FAST_STEP_PD_WORD
                 RASP_FAST_STEP_A3 RASP_FAST_STEP_B RASP_FAST_STEP_OPERANDS);
  }
  return rare;
}

// A whole epoch of fast steps as one PTX loop, run together by the lanes of
// `mask` (every lane of the mask executes it; the exits are warp-uniform).
// Each iteration is the guarded-sum step of fast_step_ptx, reorganised so
// that a step costs as few integer instructions as the case equation
// allows:
//  - the guards of every case that needs the general path (no loaded
//    instruction pair, invalid opcode, an address or jump target outside
//    [0, n), RD at the end of the tape, BNZ to itself) are evaluated first,
//    from registers only, each folded into one "leave" predicate by a
//    compare-and-combine; the end of the step count is folded into the same
//    predicate, and one warp vote leaves the loop, before anything is
//    applied, if any lane has such a step or the count is used up;
//  - otherwise every lane applies its step: the next instruction pair (at
//    the jump target or at i + 2) is loaded straight into <co, cj>, the
//    operand M[j] of ADD/MUL/PRI and the tape word of RD are loaded beside
//    it, and the opcode guards select a, the store, the output and u_0/y_0;
//  - the step countdown is not kept per step: the caller runs at most as
//    many steps as the smallest countdown of the warp;
//  - i (+) 2 is taken as ip + 2 without reduction; when that reaches ilim
//    (n, or 2^w when smaller) the next pair is not loaded, so the lane leaves
//    at its next step and the caller reduces ip. Whether the pair at the new
//    ip can be loaded (ip even and ip + 1 < ilim) is one unsigned compare of
//    ip rotated right by one bit (an odd ip sets the top bit) against
//    floor(ilim / 2).
// In: kk = steps to run (>= 1, the same in every lane of mask). Out: kk =
// steps not run; rare = 1 in the lanes whose current step needs the general
// path (nothing of it applied; 0 when the loop ended because kk reached 0);
// have = 0 when <co, cj> is not the next instruction (odd or out-of-range
// target, i (+) 2 at ilim, or overwritten by the step's own store).
// Precondition: ibase = 0, i = ip < ilim, and have = 1 only with ip even,
// ip + 1 < ilim and <co, cj> = <M[ip], M[ip+1]>.
#define RASP_LOOP_A \
      "{\n\t" \
      ".reg .pred px, pq, po, pz, pt, pe, ph, pop, p4, p6, pad, p1, p2, p3, pw, pp, pany;\n\t" \
      ".reg .b32 ol, oh, jl, jh, m, t0, t1, nip;\n\t" \
      ".reg .b64 v, tv, ado, adn, adt, ady, am;\n\t" \
      "setp.ne.u32 ph, %6, 0;\n\t" \
      "RASP_LOOP:\n\t" \
      "mov.b64 {ol, oh}, %1;\n\t" \
      "mov.b64 {jl, jh}, %2;\n\t" \
      "setp.eq.or.u32 px, %7, 0, !ph;\n\t" \
      "add.u32 t0, ol, -1;\n\t" \
      "setp.ge.or.u32 px, t0, 7, px;\n\t" \
      "setp.ne.or.u32 px, oh, 0, px;\n\t" \
      "shl.b32 m, 1, ol;\n\t"
// opcode 5's condition pz: BNZ a != 0 (word machine); BPA 1 <= a <= 2^(w-1) - 1 (classic, %17 = 2^(w-1) - 1)
#define RASP_LOOP_PZ_WORD "setp.ne.u64 pz, %0, 0;\n\t"
#define RASP_LOOP_PZ_CLASSIC "add.u64 am, %0, -1;\n\tsetp.lt.u64 pz, am, %17;\n\t"
#define RASP_LOOP_B1 \
      "setp.eq.and.u32 pt, ol, 5, pz;\n\t" \
      "setp.ge.u32 po, jl, %12;\n\t" \
      "setp.ne.or.u32 po, jh, 0, po;\n\t" \
      "and.b32 t0, m, 0xDC;\n\t" \
      "setp.ne.or.u32 pad, t0, 0, pt;\n\t"
// shared-program view: a clean VM's data access (ADD, MUL, STO, RD, PRI;
// t0 = their opcode bits) below %20 = plen takes the general path
#define RASP_LOOP_SH_GUARD \
      "setp.lt.u32 pq, jl, %20;\n\t" \
      "setp.ne.and.u32 pq, t0, 0, pq;\n\t" \
      "or.pred px, px, pq;\n\t"
#define RASP_LOOP_B2 \
      "and.pred pq, po, pad;\n\t" \
      "or.pred px, px, pq;\n\t" \
      "setp.eq.u32 p6, ol, 6;\n\t" \
      "setp.ge.and.u32 pq, %4, %14, p6;\n\t" \
      "or.pred px, px, pq;\n\t" \
      "setp.eq.and.u32 pq, jl, %3, pt;\n\t" \
      "or.pred px, px, pq;\n\t" \
      "vote.sync.any.pred pany, px, %16;\n\t" \
      "@pany bra.uni RASP_DONE;\n\t" \
      "add.u32 nip, %3, 2;\n\t" \
      "selp.b32 %3, jl, nip, pt;\n\t" \
      "shf.l.wrap.b32 t1, %3, %3, 31;\n\t" \
      "setp.lt.u32 pe, t1, %13;\n\t"
// the next instruction pair: from the slab (%9), or through a generic
// address from the code base %19 (shared-program view)
#define RASP_LOOP_ADDR_GL "mad.wide.u32 adn, %3, 8, %9;\n\t"
#define RASP_LOOP_ADDR_SH "mad.wide.u32 adn, %3, 8, %19;\n\t"
#define RASP_LOOP_B3 \
      "mad.wide.u32 ado, jl, 8, %9;\n\t" \
      "xor.b32 t1, jl, %3;\n\t" \
      "setp.eq.u32 p1, ol, 1;\n\t" \
      "@p1 mov.b64 %0, %2;\n\t"
#define RASP_LOOP_FETCH_GL "@pe ld.global.v2.u64 {%1, %2}, [adn];\n\t"
#define RASP_LOOP_FETCH_SH "@pe ld.v2.u64 {%1, %2}, [adn];\n\t"
#define RASP_LOOP_B4 \
      "and.b32 t0, m, 0x8C;\n\t" \
      "setp.ne.u32 pop, t0, 0;\n\t" \
      "@pop ld.global.u64 v, [ado];\n\t" \
      "mad.wide.u32 adt, %4, 8, %10;\n\t" \
      "@p6 ld.global.u64 tv, [adt];\n\t" \
      "setp.eq.u32 p4, ol, 4;\n\t" \
      "@p4 st.global.u64 [ado], %0;\n\t" \
      "@p6 st.global.u64 [ado], tv;\n\t" \
      "or.pred pw, p4, p6;\n\t" \
      "setp.eq.u32 p2, ol, 2;\n\t" \
      "setp.eq.u32 p3, ol, 3;\n\t" \
      "@p2 add.u64 %0, %0, v;\n\t"
#define RASP_LOOP_B RASP_LOOP_B1 RASP_LOOP_B2 RASP_LOOP_ADDR_GL RASP_LOOP_B3 RASP_LOOP_FETCH_GL RASP_LOOP_B4
// The same steps through generic addresses (M, tape and y in shared memory:
// the SMEM-staged schedule).
#define RASP_LOOP_B4_GEN \
      "and.b32 t0, m, 0x8C;\n\t" \
      "setp.ne.u32 pop, t0, 0;\n\t" \
      "@pop ld.u64 v, [ado];\n\t" \
      "mad.wide.u32 adt, %4, 8, %10;\n\t" \
      "@p6 ld.u64 tv, [adt];\n\t" \
      "setp.eq.u32 p4, ol, 4;\n\t" \
      "@p4 st.u64 [ado], %0;\n\t" \
      "@p6 st.u64 [ado], tv;\n\t" \
      "or.pred pw, p4, p6;\n\t" \
      "setp.eq.u32 p2, ol, 2;\n\t" \
      "setp.eq.u32 p3, ol, 3;\n\t" \
      "@p2 add.u64 %0, %0, v;\n\t"
#define RASP_LOOP_B_GEN RASP_LOOP_B1 RASP_LOOP_B2 RASP_LOOP_ADDR_GL RASP_LOOP_B3 RASP_LOOP_FETCH_SH RASP_LOOP_B4_GEN
#define RASP_LOOP_B_SH \
  RASP_LOOP_B1 RASP_LOOP_SH_GUARD RASP_LOOP_B2 RASP_LOOP_ADDR_SH RASP_LOOP_B3 RASP_LOOP_FETCH_SH RASP_LOOP_B4
// opcode 3 (the guards are exclusive, so each lane updates a at most once):
// MUL a * v (word machine); SUB a - v (classic)
#define RASP_LOOP_PD_WORD "@p3 mul.lo.u64 %0, %0, v;\n\t"
#define RASP_LOOP_PD_CLASSIC "@p3 sub.u64 %0, %0, v;\n\t"
#define RASP_LOOP_D \
      "setp.lt.u32 pp, %5, %15;\n\t" \
      "setp.eq.and.u32 pp, ol, 7, pp;\n\t" \
      "mad.wide.u32 ady, %5, 8, %11;\n\t" \
      "@pp st.global.u64 [ady], v;\n\t" \
      "@pp add.u32 %5, %5, 1;\n\t" \
      "@p6 add.u32 %4, %4, 1;\n\t" \
      "setp.ge.or.u32 pq, t1, 2, !pw;\n\t" \
      "and.pred ph, pe, pq;\n\t" \
      "add.u32 %7, %7, -1;\n\t" \
      "bra.uni RASP_LOOP;\n\t" \
      "RASP_DONE:\n\t" \
      "setp.ne.and.u32 px, %7, 0, px;\n\t" \
      "selp.u32 %8, 1, 0, px;\n\t" \
      "selp.u32 %6, 1, 0, ph;\n\t" \
      "}"
#define RASP_LOOP_D_GEN \
      "setp.lt.u32 pp, %5, %15;\n\t" \
      "setp.eq.and.u32 pp, ol, 7, pp;\n\t" \
      "mad.wide.u32 ady, %5, 8, %11;\n\t" \
      "@pp st.u64 [ady], v;\n\t" \
      "@pp add.u32 %5, %5, 1;\n\t" \
      "@p6 add.u32 %4, %4, 1;\n\t" \
      "setp.ge.or.u32 pq, t1, 2, !pw;\n\t" \
      "and.pred ph, pe, pq;\n\t" \
      "add.u32 %7, %7, -1;\n\t" \
      "bra.uni RASP_LOOP;\n\t" \
      "RASP_DONE:\n\t" \
      "setp.ne.and.u32 px, %7, 0, px;\n\t" \
      "selp.u32 %8, 1, 0, px;\n\t" \
      "selp.u32 %6, 1, 0, ph;\n\t" \
      "}"
#define RASP_LOOP_OPERANDS                                                                                 \
  : "+l"(a), "+l"(co), "+l"(cj), "+r"(ip), "+r"(u0), "+r"(y0), "+r"(have), "+r"(kk), "=r"(rare)             \
  : "l"(M), "l"(T), "l"(Y), "r"(n), "r"(ilim >> 1), "r"(ell), "r"(s), "r"(mask), "l"(wmask >> 1),           \
    "l"(wmask)                                                                                               \
  : "memory"

template <bool MASKED, bool CLASSIC>
__device__ __forceinline__ uint32_t fast_loop_ptx(uint64_t* M, const uint64_t* T, uint64_t* Y, uint32_t n,
                                                  uint32_t ell, uint32_t s, uint32_t ilim, uint64_t wmask,
                                                  uint32_t mask, uint64_t& a, uint64_t& co, uint64_t& cj,
                                                  uint32_t& ip, uint32_t& u0, uint32_t& y0, uint32_t& have,
                                                  uint32_t& kk) {
  uint32_t rare;
  // w < 64: the new accumulator is reduced to w bits (%18 = 2^w - 1)
  if constexpr (MASKED && CLASSIC) {
    asm volatile(RASP_LOOP_A RASP_LOOP_PZ_CLASSIC RASP_LOOP_B RASP_LOOP_PD_CLASSIC
                 "and.b64 %0, %0, %18;\n\t" RASP_LOOP_D RASP_LOOP_OPERANDS);
  } else if constexpr (MASKED) {
    asm volatile(RASP_LOOP_A RASP_LOOP_PZ_WORD RASP_LOOP_B RASP_LOOP_PD_WORD
                 "and.b64 %0, %0, %18;\n\t" RASP_LOOP_D RASP_LOOP_OPERANDS);
  } else if constexpr (CLASSIC) {
    asm volatile(RASP_LOOP_A RASP_LOOP_PZ_CLASSIC RASP_LOOP_B RASP_LOOP_PD_CLASSIC RASP_LOOP_D
                 RASP_LOOP_OPERANDS);
  } else {
    asm volatile(RASP_LOOP_A RASP_LOOP_PZ_WORD RASP_LOOP_B RASP_LOOP_PD_WORD RASP_LOOP_D
                 RASP_LOOP_OPERANDS);
  }
  return rare;
}

// The epoch loop of the SMEM-staged schedule: the steps of fast_loop_ptx
// with every access through a generic address (M, the tape and y of the lane
// sit in shared memory). Word opcode set, w = 64 or masked.
template <bool MASKED>
__device__ __forceinline__ uint32_t fast_loop_ptx_gen(uint64_t* M, const uint64_t* T, uint64_t* Y, uint32_t n,
                                                      uint32_t ell, uint32_t s, uint32_t ilim, uint64_t wmask,
                                                      uint32_t mask, uint64_t& a, uint64_t& co, uint64_t& cj,
                                                      uint32_t& ip, uint32_t& u0, uint32_t& y0, uint32_t& have,
                                                      uint32_t& kk) {
  uint32_t rare;
  if constexpr (MASKED) {
    asm volatile(RASP_LOOP_A RASP_LOOP_PZ_WORD RASP_LOOP_B_GEN RASP_LOOP_PD_WORD
                 "and.b64 %0, %0, %18;\n\t" RASP_LOOP_D_GEN RASP_LOOP_OPERANDS);
  } else {
    asm volatile(RASP_LOOP_A RASP_LOOP_PZ_WORD RASP_LOOP_B_GEN RASP_LOOP_PD_WORD RASP_LOOP_D_GEN
                 RASP_LOOP_OPERANDS);
  }
  return rare;
}

// The epoch loop for a VM seen through a shared-program view (word opcode
// set): instruction pairs are loaded through a generic address from the
// code base `code` (the program in shared memory while the VM is clean, else
// its slab), `ilim` is the fetch limit (min(plen, ilim) while clean), and a
// data access below `dlo` (plen while clean, else 0) takes the general path,
// so that every data access in the loop goes to the slab.
#define RASP_LOOP_SH_OPERANDS                                                                              \
  : "+l"(a), "+l"(co), "+l"(cj), "+r"(ip), "+r"(u0), "+r"(y0), "+r"(have), "+r"(kk), "=r"(rare)             \
  : "l"(M), "l"(T), "l"(Y), "r"(n), "r"(ilim >> 1), "r"(ell), "r"(s), "r"(mask), "l"(wmask >> 1),           \
    "l"(wmask), "l"(code), "r"(dlo)                                                                          \
  : "memory"

template <bool MASKED>
__device__ __forceinline__ uint32_t fast_loop_ptx_sh(uint64_t* M, const uint64_t* code, uint32_t dlo,
                                                     const uint64_t* T, uint64_t* Y, uint32_t n, uint32_t ell,
                                                     uint32_t s, uint32_t ilim, uint64_t wmask, uint32_t mask,
                                                     uint64_t& a, uint64_t& co, uint64_t& cj, uint32_t& ip,
                                                     uint32_t& u0, uint32_t& y0, uint32_t& have, uint32_t& kk) {
  uint32_t rare;
  if constexpr (MASKED) {
    asm volatile(RASP_LOOP_A RASP_LOOP_PZ_WORD RASP_LOOP_B_SH RASP_LOOP_PD_WORD
                 "and.b64 %0, %0, %18;\n\t" RASP_LOOP_D RASP_LOOP_SH_OPERANDS);
  } else {
    asm volatile(RASP_LOOP_A RASP_LOOP_PZ_WORD RASP_LOOP_B_SH RASP_LOOP_PD_WORD RASP_LOOP_D
                 RASP_LOOP_SH_OPERANDS);
  }
  return rare;
}

// The epoch loop of a narrow batch (w <= 32, M in 4-byte words): the same
// steps as fast_loop_ptx with 32-bit words and 32-bit arithmetic (every word
// and a are below 2^w <= 2^32, so a word's high half is never looked at and
// the sum and product are taken mod 2^32, then reduced to w bits when
// w < 32). Tape words and outputs stay 8-byte words whose high halves are
// zero: RD reads a tape word's low half, PRI writes an output's low half.
// a, co and cj are 32-bit here; the caller widens them.
#define RASP_NLOOP_A \
      "{\n\t" \
      ".reg .pred px, pq, po, pz, pt, pe, ph, pop, p4, p6, pad, p1, p2, p3, pw, pp, pany;\n\t" \
      ".reg .b32 m, t0, t1, nip, v, tv, am, jl, ol;\n\t" \
      ".reg .b64 ado, adn, adt, ady;\n\t" \
      "setp.ne.u32 ph, %6, 0;\n\t" \
      "RASP_NLOOP:\n\t" \
      "mov.b32 ol, %1;\n\t" \
      "mov.b32 jl, %2;\n\t" \
      "setp.eq.or.u32 px, %7, 0, !ph;\n\t" \
      "add.u32 t0, ol, -1;\n\t" \
      "setp.ge.or.u32 px, t0, 7, px;\n\t" \
      "shl.b32 m, 1, ol;\n\t"
#define RASP_NLOOP_PZ_WORD "setp.ne.u32 pz, %0, 0;\n\t"
#define RASP_NLOOP_PZ_CLASSIC "add.u32 am, %0, -1;\n\tsetp.lt.u32 pz, am, %17;\n\t"
#define RASP_NLOOP_B \
      "setp.eq.and.u32 pt, ol, 5, pz;\n\t" \
      "setp.ge.u32 po, jl, %12;\n\t" \
      "and.b32 t0, m, 0xDC;\n\t" \
      "setp.ne.or.u32 pad, t0, 0, pt;\n\t" \
      "and.pred pq, po, pad;\n\t" \
      "or.pred px, px, pq;\n\t" \
      "setp.eq.u32 p6, ol, 6;\n\t" \
      "setp.ge.and.u32 pq, %4, %14, p6;\n\t" \
      "or.pred px, px, pq;\n\t" \
      "setp.eq.and.u32 pq, jl, %3, pt;\n\t" \
      "or.pred px, px, pq;\n\t" \
      "vote.sync.any.pred pany, px, %16;\n\t" \
      "@pany bra.uni RASP_NDONE;\n\t" \
      "add.u32 nip, %3, 2;\n\t" \
      "selp.b32 %3, jl, nip, pt;\n\t" \
      "shf.l.wrap.b32 t1, %3, %3, 31;\n\t" \
      "setp.lt.u32 pe, t1, %13;\n\t" \
      "mad.wide.u32 adn, %3, 4, %9;\n\t" \
      "mad.wide.u32 ado, jl, 4, %9;\n\t" \
      "xor.b32 t1, jl, %3;\n\t" \
      "setp.eq.u32 p1, ol, 1;\n\t" \
      "@p1 mov.b32 %0, jl;\n\t" \
      "@pe ld.global.v2.u32 {%1, %2}, [adn];\n\t" \
      "and.b32 t0, m, 0x8C;\n\t" \
      "setp.ne.u32 pop, t0, 0;\n\t" \
      "@pop ld.global.u32 v, [ado];\n\t" \
      "mad.wide.u32 adt, %4, 8, %10;\n\t" \
      "@p6 ld.global.u32 tv, [adt];\n\t" \
      "setp.eq.u32 p4, ol, 4;\n\t" \
      "@p4 st.global.u32 [ado], %0;\n\t" \
      "@p6 st.global.u32 [ado], tv;\n\t" \
      "or.pred pw, p4, p6;\n\t" \
      "setp.eq.u32 p2, ol, 2;\n\t" \
      "setp.eq.u32 p3, ol, 3;\n\t" \
      "@p2 add.u32 %0, %0, v;\n\t"
#define RASP_NLOOP_PD_WORD "@p3 mul.lo.u32 %0, %0, v;\n\t"
#define RASP_NLOOP_PD_CLASSIC "@p3 sub.u32 %0, %0, v;\n\t"
#define RASP_NLOOP_D \
      "setp.lt.u32 pp, %5, %15;\n\t" \
      "setp.eq.and.u32 pp, ol, 7, pp;\n\t" \
      "mad.wide.u32 ady, %5, 8, %11;\n\t" \
      "@pp st.global.u32 [ady], v;\n\t" \
      "@pp add.u32 %5, %5, 1;\n\t" \
      "@p6 add.u32 %4, %4, 1;\n\t" \
      "setp.ge.or.u32 pq, t1, 2, !pw;\n\t" \
      "and.pred ph, pe, pq;\n\t" \
      "add.u32 %7, %7, -1;\n\t" \
      "bra.uni RASP_NLOOP;\n\t" \
      "RASP_NDONE:\n\t" \
      "setp.ne.and.u32 px, %7, 0, px;\n\t" \
      "selp.u32 %8, 1, 0, px;\n\t" \
      "selp.u32 %6, 1, 0, ph;\n\t" \
      "}"
#define RASP_NLOOP_OPERANDS                                                                                \
  : "+r"(a), "+r"(co), "+r"(cj), "+r"(ip), "+r"(u0), "+r"(y0), "+r"(have), "+r"(kk), "=r"(rare)             \
  : "l"(M), "l"(T), "l"(Y), "r"(n), "r"(ilim >> 1), "r"(ell), "r"(s), "r"(mask), "r"(wmask >> 1),           \
    "r"(wmask)                                                                                               \
  : "memory"

// MASK: w < 32 (the new accumulator is reduced to w bits, %18 = 2^w - 1).
template <bool MASK, bool CLASSIC>
__device__ __forceinline__ uint32_t fast_loop_ptx_narrow(uint32_t* M, const uint64_t* T, uint64_t* Y, uint32_t n,
                                                         uint32_t ell, uint32_t s, uint32_t ilim, uint32_t wmask,
                                                         uint32_t mask, uint32_t& a, uint32_t& co, uint32_t& cj,
                                                         uint32_t& ip, uint32_t& u0, uint32_t& y0, uint32_t& have,
                                                         uint32_t& kk) {
  uint32_t rare;
  if constexpr (MASK && CLASSIC) {
    asm volatile(RASP_NLOOP_A RASP_NLOOP_PZ_CLASSIC RASP_NLOOP_B RASP_NLOOP_PD_CLASSIC
                 "and.b32 %0, %0, %18;\n\t" RASP_NLOOP_D RASP_NLOOP_OPERANDS);
  } else if constexpr (MASK) {
    asm volatile(RASP_NLOOP_A RASP_NLOOP_PZ_WORD RASP_NLOOP_B RASP_NLOOP_PD_WORD
                 "and.b32 %0, %0, %18;\n\t" RASP_NLOOP_D RASP_NLOOP_OPERANDS);
  } else if constexpr (CLASSIC) {
    asm volatile(RASP_NLOOP_A RASP_NLOOP_PZ_CLASSIC RASP_NLOOP_B RASP_NLOOP_PD_CLASSIC RASP_NLOOP_D
                 RASP_NLOOP_OPERANDS);
  } else {
    asm volatile(RASP_NLOOP_A RASP_NLOOP_PZ_WORD RASP_NLOOP_B RASP_NLOOP_PD_WORD RASP_NLOOP_D
                 RASP_NLOOP_OPERANDS);
  }
  return rare;
}

template <bool MASKED, bool CHECKED, bool HIST, bool PIPE, bool CLASSIC = false, class Mem>
__device__ __forceinline__ uint32_t one_step(Mem M, const uint64_t* __restrict__ T, uint64_t* __restrict__ Y,
                                             const Params& P, Regs& r, Hist& h) {
  const uint32_t ip = r.ip, n = r.n;
  if constexpr (PIPE && !CHECKED && !HIST && std::is_pointer<Mem>::value) {
    if (r.have) {
      uint64_t co = r.cur.x, cj = r.cur.y;
      uint32_t hv = 1;
      const uint32_t rare = fast_step_ptx<MASKED, CLASSIC>(M, T, Y, n, P.ell, P.s, r.a, co, cj, r.ip, r.left,
                                                           r.u0, r.y0, hv, MASKED ? r.ilim : n, P.wmask);
      if (!rare) {
        r.cur.x = co;
        r.cur.y = cj;
        r.have = hv != 0u;
        return CONT;
      }
    }
    r.have = false;
    const uint32_t s = step_general<MASKED, CHECKED, HIST, CLASSIC>(M, T, Y, P, r, h);
    if (s == CONT) prime(M, r);
    return s;
  }
  const uint32_t ilim = MASKED ? r.ilim : n;
  // i = ip < n even with ip + 1 < n: i != 2^w - 1 and M[ip], M[ip+1] is one
  // aligned 16-byte word (slabs start 16-byte aligned)
  const bool aligned = ((ip & 1u) == 0u) & (ip + 1u < n) & (r.ibase == 0ull);
  if (PIPE && aligned && !r.have) {
    r.cur = mem_pair(M, r.clean, ip);
    r.have = true;
  }
  if (aligned) {
    // (a shared-program view serves a clean VM's code words from the one
    // copy of the program in shared memory)
    const ulonglong2 oj = PIPE ? r.cur : mem_pair(M, r.clean, ip);
    const uint64_t o = oj.x, j = oj.y, a = r.a;
    const uint32_t op = (uint32_t)o, jm = (uint32_t)j;
    const bool valid = (o - 1ull) < 7ull;
    const bool jin = j < (uint64_t)n;
    const bool taken = (op == 5u) & jumps<CLASSIC>(a, MASKED ? P.wmask : ~0ull);
    const bool rd = op == 6u;
    const bool pri = op == 7u;
    const bool seq_ok = ip + 3u < n;
    ulonglong2 seq = make_ulonglong2(0ull, 0ull);
    ulonglong2 pr = make_ulonglong2(0ull, 0ull);
    uint64_t v = 0;
    if (PIPE) {
      if (seq_ok) seq = mem_pair(M, r.clean, ip + 2u);
      if (((op == 2u) | (op == 3u) | pri | taken) & jin) pr = mem_pair(M, r.clean, jm & ~1u);
      v = (jm & 1u) ? pr.y : pr.x;
    } else {
      if (((op == 2u) | (op == 3u) | pri) & jin) v = mem_rd(M, r.clean, jm);
    }
    const uint64_t sum = a + v;
    const uint64_t prod = CLASSIC ? a - v : a * v;       // opcode 3: MUL, or SUB in the classic set
    const bool addr = ((op >= 2u) & (op != 5u)) | taken;   // j used as an address or jump target
    // rare: invalid opcode, operand outside memory, countdown exhausted, RD at
    // the end of the tape, BNZ to itself, i (+) 2 at the end of memory or 2^w
    bool rare = !valid | (addr & !jin) | (r.left == 0u) | (rd & (r.u0 >= P.ell)) |
                (taken ? (jm == ip) : (ip + 2u >= ilim));
    if constexpr (CHECKED) {
      rare |= (op == 2u) & ((int64_t)((a ^ sum) & (v ^ sum)) < 0);
      if constexpr (CLASSIC) rare |= (op == 3u) & ((int64_t)((a ^ v) & (a ^ prod)) < 0);
      else rare |= (op == 3u) & (__mul64hi((long long)a, (long long)v) != ((int64_t)prod >> 63));
    }
    if (!rare) {
      uint64_t na = (op == 1u) ? j : a;
      na = (op == 2u) ? sum : na;
      na = (op == 3u) ? prod : na;
      if (MASKED) na &= P.wmask;
      const bool wr = (op == 4u) | rd;
      uint64_t w = a;                            // STO writes a, RD writes u-bullet
      if (rd) w = T[r.u0];
      if (wr) mem_wr(M, r.clean, jm, w);
      const bool put = pri & (r.y0 < P.s);       // y :: M_{j mod n}
      if (put) Y[r.y0] = v;
      r.u0 += rd ? 1u : 0u;
      r.y0 += put ? 1u : 0u;
      r.a = na;
      const uint32_t nip = taken ? jm : ip + 2u;
      r.ip = nip;
      if (PIPE) {
        // the next pair: the jump target's (if aligned) or the sequential one,
        // unless this step's store overwrote it
        r.cur = taken ? pr : seq;
        r.have = taken ? (((jm & 1u) == 0u) & (jm + 1u < n)) : (seq_ok & !(wr & ((jm | 1u) == (nip | 1u))));
      }
      r.left -= 1u;
      if constexpr (HIST) h.c[8] += (pri & !put) ? 1u : 0u;
      count_step<HIST>(h, op, taken);
      return CONT;
    }
  }
  if (PIPE) r.have = false;
  return step_general<MASKED, CHECKED, HIST, CLASSIC>(M, T, Y, P, r, h);
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

// Registers of VM v, read from the state store (i goes to ibase until
// arm_regs splits it).
__device__ __forceinline__ void load_regs(const DevState& S, const Params& P, uint32_t v, Regs& r) {
  r.ibase = S.i[v];
  r.a = S.a[v];
  r.steps = S.steps[v];
  r.cap = S.cap[v];
  r.n = S.n[v];
  r.u0 = S.uhead[v];
  r.y0 = S.ylen[v];
}

// Derived registers once the loads of load_regs have landed.
__device__ __forceinline__ void arm_regs(const Params& P, Regs& r) {
  const uint64_t i = r.ibase;
  r.ip = mod_n(i, r.n);
  r.ibase = i - r.ip;
  r.ilim = (P.wmask >= (uint64_t)r.n - 1u) ? r.n : (uint32_t)(P.wmask + 1ull);
  r.have = false;
  arm_countdown(P, r);
}

__device__ __forceinline__ void store_regs(const DevState& S, uint32_t v, const Regs& r, uint32_t st) {
  S.i[v] = i_of(r);
  S.a[v] = r.a;
  S.steps[v] = steps_of(r);
  S.uhead[v] = r.u0;
  S.ylen[v] = r.y0;
  S.status[v] = (uint8_t)st;
}

}  // namespace rasp
