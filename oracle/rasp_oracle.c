/*
 * rasp_oracle.c -- serial CPU oracle for the word RASP  R^(w,n,l,s).
 *
 * TEST INFRASTRUCTURE. This is the plain, slow, obviously correct statement
 * of what the batched GPU engine computes. Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load it; the product path never
 * does. It shares no code, header, table or helper with the CUDA path.
 *
 * Paper: B. Considine, "Towards a Linear-Algebraic Hypervisor".
 *   Sec. 2.1  configuration space  C_w = W x W x W^n x W^(l+1) x W^(s+1),
 *             c = <i, a, M, u, y>;
 *   Sec. 2.1  initial configuration  c_0(P, x) = <0, 0, P 0^(n-2m), x 0^(l-|x|), 0^(s+1)>;
 *   Sec. 2.1  (+) and (x) modulo 2^w; circular addressing
 *             <o, j> = <M[i mod n], M[(i (+) 1) mod n]>; the operators
 *             M_j <- a, u-bullet, u-triangle and y :: z;
 *   Sec. 2.1  the one-step transition (case equation, opcodes 1 LOD .. 7 PRI,
 *             "otherwise" = identity) and the halting set F = {c : c -> c};
 *   Sec. 3    halting number tau_h = least tau with Phi^tau(c0) = Phi^(tau+1)(c0).
 *   Sec. 1.1  the classic RASP opcode set, selected by `isa`: opcode 3 is SUB
 *             (a - M_j) and opcode 5 is BPA (jump when a > 0); the word
 *             machine of Sec. 2.1 has MUL and BNZ there.
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *   - u[0] is the read head and u[1..l] the zero-padded input; y[0] is the
 *     output count and y[1..s] the output words (the W^(l+1), W^(s+1) shapes).
 *   - Words are bit vectors: "x mod n" uses the unsigned value of x.
 *   - i is a full w-bit word and is never reduced; only the fetch index is.
 *   - LOD is immediate: a <- j.
 *   - A VM is HALTED as soon as its configuration is a fixed point. The fixed
 *     point test here is literal equality of c and its successor; the
 *     successor differs from c only in the fields recorded in `succ`, so
 *     comparing those fields is comparing the whole tuple.
 *   - steps counts applied (state-changing) transitions, so steps = tau_h for
 *     a halted VM. When steps reaches min(budget, cap) the VM is HALTED if it
 *     is a fixed point there, else TIMEOUT if steps == cap, else it stays
 *     RUNNING (a later call with a larger budget resumes it).
 *   - CHECKED semantics (no counterpart in the paper; parity unpinned by the
 *     paper): memory is not circular and arithmetic is signed 64-bit.
 *     Order: (1) fetch range, i in [0, n-1) else FAULT_ADDR; (2) fixed point
 *     -> HALTED; (3) operand range, j in [0, n) for ADD, MUL/SUB, STO, PRI and
 *     for RD when it fires, else FAULT_ADDR; (4) signed overflow of ADD or
 *     MUL/SUB -> FAULT_OVERFLOW. A faulting step is neither applied nor counted.
 *   - Classic opcode set on w-bit words (Sec. 1.1 states it over the
 *     integers): SUB is a - M_j modulo 2^w, and BPA's "a > 0" reads the w-bit
 *     word a as a two's complement integer, so it jumps iff
 *     1 <= a <= 2^(w-1) - 1. Everything else is the word machine's.
 */
#include <stdint.h>
#include <stddef.h>

enum { RO_RUNNING = 0, RO_HALTED = 1, RO_TIMEOUT = 2,
       RO_FAULT_OVERFLOW = 3, RO_FAULT_ADDR = 4 };

enum { RO_OK = 0, RO_EINVAL = -1 };

/* Machine parameters shared by a batch. */
typedef struct {
    uint32_t w;        /* word bits, 1..64                         */
    uint32_t checked;  /* 0: the paper's wrapping machine, 1: CHECKED */
    uint64_t ell;      /* l, input tape capacity                    */
    uint64_t s;        /* s, output tape capacity                   */
    uint32_t isa;      /* RO_ISA_WORD (Sec. 2.1) or RO_ISA_CLASSIC (Sec. 1.1) */
    uint32_t pad;
} ro_params;

enum { RO_ISA_WORD = 0, RO_ISA_CLASSIC = 1 };

/* One machine, viewed in place. */
typedef struct {
    uint64_t *i, *a;
    uint64_t *M; uint64_t n;
    uint64_t *u;       /* l+1 words: u[0] head, u[1..l] tape   */
    uint64_t *y;       /* s+1 words: y[0] count, y[1..s] data  */
} ro_vm;

/* The successor c' of c, as the fields that a transition may change. */
typedef struct {
    uint64_t op;                   /* opcode o that was fetched          */
    uint64_t i, a, u0, y0;
    int m_set; uint64_t m_idx, m_val;   /* M_k <- value               */
    int y_set; uint64_t y_idx, y_val;   /* y_k <- value               */
} ro_succ;

static uint64_t word_mask(uint32_t w) {
    return w >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << w) - 1);
}

static uint64_t min_u64(uint64_t x, uint64_t y) { return x < y ? x : y; }

/* Does opcode 5 jump? BNZ: a != 0. BPA: a > 0, with a read as a w-bit two's
   complement integer (its top bit w-1 is the sign). */
static int branch_taken(const ro_params *p, uint64_t a) {
    if (p->isa != RO_ISA_CLASSIC) return a != 0;
    const int negative = (int)((a >> (p->w - 1)) & 1);
    return a != 0 && !negative;
}

/* c -> c' (Sec. 2.1 case equation), wrapping semantics. */
static void successor(const ro_params *p, const ro_vm *c, ro_succ *s) {
    const uint64_t mask = word_mask(p->w);
    const uint64_t i = *c->i, a = *c->a, n = c->n;
    const uint64_t o = c->M[i % n];                    /* M_{i mod n}         */
    const uint64_t j = c->M[((i + 1) & mask) % n];     /* M_{(i (+) 1) mod n} */
    const uint64_t i_next = (i + 2) & mask;            /* i (+) 2             */
    const uint64_t k = j % n;                          /* j mod n             */

    s->op = o;
    s->i = i; s->a = a; s->u0 = c->u[0]; s->y0 = c->y[0];
    s->m_set = 0; s->m_idx = 0; s->m_val = 0;
    s->y_set = 0; s->y_idx = 0; s->y_val = 0;

    switch (o) {
    case 1:  /* LOD: <i (+) 2, j, M, u, y> */
        s->i = i_next; s->a = j;
        break;
    case 2:  /* ADD: <i (+) 2, a (+) M_{j mod n}, M, u, y> */
        s->i = i_next; s->a = (a + c->M[k]) & mask;
        break;
    case 3:
        if (p->isa == RO_ISA_CLASSIC) {   /* SUB: <i (+) 2, a - M_{j mod n}, M, u, y> */
            s->i = i_next; s->a = (a - c->M[k]) & mask;
        } else {                          /* MUL: <i (+) 2, a (x) M_{j mod n}, M, u, y> */
            s->i = i_next; s->a = (a * c->M[k]) & mask;
        }
        break;
    case 4:  /* STO: <i (+) 2, a, M_{j mod n} <- a, u, y> */
        s->i = i_next;
        s->m_set = 1; s->m_idx = k; s->m_val = a;
        break;
    case 5:  /* BNZ (BPA): <j, a, M, u, y> if a != 0 (a > 0), else <i (+) 2, a, M, u, y> */
        s->i = branch_taken(p, a) ? j : i_next;
        break;
    case 6:  /* RD, only when u_0 < l:
                <i (+) 2, a, M_{j mod n} <- u-bullet, u-triangle, y> */
        if (c->u[0] < p->ell) {
            s->i = i_next;
            s->m_set = 1; s->m_idx = k;
            s->m_val = c->u[min_u64(c->u[0] + 1, p->ell)];  /* u-bullet   */
            s->u0 = min_u64(c->u[0] + 1, p->ell);           /* u-triangle */
        }
        break;
    case 7:  /* PRI: <i (+) 2, a, M, u, y :: M_{j mod n}> */
        s->i = i_next;
        if (c->y[0] < p->s) {
            s->y_set = 1; s->y_idx = c->y[0] + 1; s->y_val = c->M[k];
            s->y0 = c->y[0] + 1;
        }
        break;
    default: /* otherwise: <i, a, M, u, y> */
        break;
    }
}

/* c' == c ? (F = {c : c -> c}) */
static int is_fixed(const ro_vm *c, const ro_succ *s) {
    if (s->i != *c->i || s->a != *c->a) return 0;
    if (s->u0 != c->u[0] || s->y0 != c->y[0]) return 0;
    if (s->m_set && c->M[s->m_idx] != s->m_val) return 0;
    if (s->y_set && c->y[s->y_idx] != s->y_val) return 0;
    return 1;
}

static void apply(ro_vm *c, const ro_succ *s) {
    if (s->m_set) c->M[s->m_idx] = s->m_val;
    if (s->y_set) c->y[s->y_idx] = s->y_val;
    *c->i = s->i; *c->a = s->a;
    c->u[0] = s->u0; c->y[0] = s->y0;
}

enum { K_APPLY = 0, K_FIXED = 1, K_FAULT_ADDR = 2, K_FAULT_OVERFLOW = 3 };

/* What the next transition of c would do, including the CHECKED faults. */
static int classify(const ro_params *p, const ro_vm *c, ro_succ *s) {
    if (p->checked) {
        const uint64_t i = *c->i;
        if (!(i < c->n - 1)) {            /* fetch needs i and i+1 in [0, n) */
            s->op = 0;
            return K_FAULT_ADDR;
        }
    }
    successor(p, c, s);
    if (is_fixed(c, s)) return K_FIXED;
    if (p->checked) {
        const uint64_t o = s->op;
        const uint64_t j = c->M[*c->i + 1];
        const int uses_address = (o == 2 || o == 3 || o == 4 || o == 7 ||
                                  (o == 6 && c->u[0] < p->ell));
        if (uses_address && !(j < c->n)) return K_FAULT_ADDR;
        if (o == 2 || o == 3) {
            const int64_t x = (int64_t)*c->a, y = (int64_t)c->M[j];
            int64_t r;
            const int ovf = (o == 2) ? __builtin_add_overflow(x, y, &r)
                          : (p->isa == RO_ISA_CLASSIC) ? __builtin_sub_overflow(x, y, &r)
                                                       : __builtin_mul_overflow(x, y, &r);
            if (ovf) return K_FAULT_OVERFLOW;
        }
    }
    return K_APPLY;
}

/*
 * Pack c_0(P, x) for `count` machines (Sec. 2.1).
 *   n[v]          memory words of VM v (n >= 1)
 *   mem_off[v]    offset of VM v's M in `mem`
 *   prog, prog_off[count+1]   program words of VM v: prog[prog_off[v] .. prog_off[v+1])
 *   tape, tape_off[count+1]   input x of VM v
 * Output: mem, i, a (zeroed), u [count*(l+1)], y [count*(s+1)], steps, status.
 * Program and input words are reduced to w bits. Returns RO_EINVAL if a
 * program has odd length or 2m > n, or an input is longer than l.
 */
int ro_pack(const ro_params *p, uint64_t count,
            const uint64_t *n, const uint64_t *mem_off, uint64_t *mem,
            const uint64_t *prog, const uint64_t *prog_off,
            const uint64_t *tape, const uint64_t *tape_off,
            uint64_t *i, uint64_t *a, uint64_t *u, uint64_t *y,
            uint64_t *steps, uint8_t *status) {
    const uint64_t mask = word_mask(p->w);
    if (p->w < 1 || p->w > 64) return RO_EINVAL;
    if (p->checked && p->w != 64) return RO_EINVAL;
    for (uint64_t v = 0; v < count; ++v) {
        const uint64_t plen = prog_off[v + 1] - prog_off[v];
        const uint64_t xlen = tape_off[v + 1] - tape_off[v];
        if (n[v] < 1 || (plen & 1) || plen > n[v] || xlen > p->ell) return RO_EINVAL;
        uint64_t *M = mem + mem_off[v];
        for (uint64_t k = 0; k < n[v]; ++k)
            M[k] = (k < plen) ? (prog[prog_off[v] + k] & mask) : 0;
        uint64_t *uv = u + v * (p->ell + 1);
        uv[0] = 0;
        for (uint64_t k = 0; k < p->ell; ++k)
            uv[1 + k] = (k < xlen) ? (tape[tape_off[v] + k] & mask) : 0;
        uint64_t *yv = y + v * (p->s + 1);
        for (uint64_t k = 0; k <= p->s; ++k) yv[k] = 0;
        i[v] = 0; a[v] = 0; steps[v] = 0; status[v] = RO_RUNNING;
    }
    return RO_OK;
}

/*
 * Advance machines [first, first+count) until each is no longer RUNNING or
 * has taken min(budget, cap[v]) steps in total (steps is cumulative).
 * hist (optional, 9 entries) accumulates applied steps by opcode 1..7;
 * hist[8] counts PRI steps that found the output tape full, hist[0] the
 * taken BNZ steps.
 */
int ro_run(const ro_params *p, uint64_t first, uint64_t count,
           const uint64_t *n, const uint64_t *mem_off, uint64_t *mem,
           uint64_t *i, uint64_t *a, uint64_t *u, uint64_t *y,
           uint64_t *steps, const uint64_t *cap, uint8_t *status,
           uint64_t budget, uint64_t *hist) {
    if (p->w < 1 || p->w > 64) return RO_EINVAL;
    if (p->checked && p->w != 64) return RO_EINVAL;
    for (uint64_t v = first; v < first + count; ++v) {
        if (status[v] != RO_RUNNING) continue;
        ro_vm c;
        c.i = &i[v]; c.a = &a[v];
        c.M = mem + mem_off[v]; c.n = n[v];
        c.u = u + v * (p->ell + 1);
        c.y = y + v * (p->s + 1);
        const uint64_t stop = min_u64(budget, cap[v]);
        for (;;) {
            ro_succ s;
            const int kind = classify(p, &c, &s);
            if (kind == K_FIXED) { status[v] = RO_HALTED; break; }
            if (steps[v] >= stop) {
                status[v] = (steps[v] >= cap[v]) ? RO_TIMEOUT : RO_RUNNING;
                break;
            }
            if (kind == K_FAULT_ADDR) { status[v] = RO_FAULT_ADDR; break; }
            if (kind == K_FAULT_OVERFLOW) { status[v] = RO_FAULT_OVERFLOW; break; }
            if (hist) {
                hist[s.op] += 1;
                if (s.op == 7 && !s.y_set) hist[8] += 1;
                if (s.op == 5 && branch_taken(p, *c.a)) hist[0] += 1;
            }
            apply(&c, &s);
            steps[v] += 1;
        }
    }
    return RO_OK;
}

/* Single transition of one machine, for tests: returns the classification
   (0 apply, 1 fixed, 2 address fault, 3 overflow fault) and applies it when
   it is 0. */
int ro_step_one(const ro_params *p, uint64_t *i, uint64_t *a,
                uint64_t *M, uint64_t n, uint64_t *u, uint64_t *y) {
    ro_vm c = { i, a, M, n, u, y };
    ro_succ s;
    const int kind = classify(p, &c, &s);
    if (kind == K_APPLY) apply(&c, &s);
    return kind;
}
