/*
 * progsampler.c -- the program sampler of sampler.py, in C, for speed.
 *
 * Input generation only: it draws programs of the array language uniformly
 * by token length (the halting experiment of "Towards a Linear-Algebraic
 * Hypervisor", Sec. 3), lowers them by the rules of Sec. 2.2 and draws their
 * input tapes. It holds none of the machine's arithmetic. It is a
 * transcription of the Python definition in sampler.py / dsl.py and must
 * produce identical words: the same Philox4x32-10 draws (Salmon et al.,
 * SC'11) consumed in the same order, the same cumulative probability tables
 * (computed in Python from exact counts and passed in), the same lowering.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox */
static void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint64_t p0 = (uint64_t)c[0] * 0xD2511F53u;
        const uint64_t p1 = (uint64_t)c[2] * 0xCD9E8D57u;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

/* word k of stream (seed, tag, id): counter (k / 4, id_lo, id_hi, tag),
   key (seed_lo, seed_hi), lane k % 4 */
static uint32_t draw(uint64_t seed, uint32_t tag, uint64_t id, uint32_t k) {
    uint32_t c[4] = {k / 4, (uint32_t)id, (uint32_t)(id >> 32), tag};
    philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return c[k % 4];
}

/* sequential draws of one program: 64-word blocks, block b from tag0 + b */
typedef struct {
    uint64_t seed, id;
    uint32_t tag0, block, pos;
    uint32_t buf[4];
    uint32_t buf_ctr;      /* counter (pos / 4) held in buf, or ~0 */
} stream;

static uint32_t word(stream *s) {
    if (s->pos == 64) { s->block++; s->pos = 0; s->buf_ctr = ~0u; }
    const uint32_t ctr = s->pos / 4;
    if (ctr != s->buf_ctr) {
        uint32_t c[4] = {ctr, (uint32_t)s->id, (uint32_t)(s->id >> 32), s->tag0 + s->block};
        philox10(c, (uint32_t)s->seed, (uint32_t)(s->seed >> 32));
        memcpy(s->buf, c, sizeof(c));
        s->buf_ctr = ctr;
    }
    return s->buf[s->pos++ % 4];
}

static double uniform(stream *s) {
    const uint64_t a = word(s) >> 5;
    const uint64_t b = word(s) >> 6;
    return (double)(a * 67108864u + b) / 9007199254740992.0;
}

static uint32_t below(stream *s, uint32_t k) { return (uint32_t)(((uint64_t)word(s) * k) >> 32); }

/* ---------------------------------------------------------------- tables */
/* Alternatives of S and B at each length l: entries [off[l], off[l+1]) of
   cum (cumulative probability), kind, a, b.
   S kinds: 0 put (a = |E|), 1 ife (a = |B1|, b = |B2|), 2 whl (a = |B|).
   B kinds: 0 the block is one statement (of length l), 1 hlt, 2 S ; B
   (a = |S|, b = |B|). */
typedef struct {
    uint32_t L;
    const uint32_t *s_off; const double *s_cum; const int32_t *s_kind, *s_a, *s_b;
    const uint32_t *b_off; const double *b_cum; const int32_t *b_kind, *b_a, *b_b;
} gen_tables;

static uint32_t pick(stream *s, const uint32_t *off, const double *cum, uint32_t l) {
    const uint32_t lo = off[l], hi = off[l + 1];
    if (hi - lo <= 1) return lo;                 /* one alternative: no draw */
    const double u = uniform(s);
    uint32_t k = lo;                             /* bisect_right: entries <= u */
    while (k < hi && cum[k] <= u) ++k;
    return k;
}

/* ---------------------------------------------------------------- AST */
enum { ST_HLT = 0, ST_PUT = 1, ST_IFE = 2, ST_WHL = 3 };
enum { EX_CONST = 0, EX_GET = 1, EX_BIN = 2 };
enum { AR_IPT = 0, AR_SCR = 1, AR_OPT = 2 };     /* GET arrays order: ipt, scr, opt */

typedef struct { int32_t arr, z; } ref;
typedef struct { int32_t kind, op; ref g; int32_t c; ref h; int32_t rhs_const; } expr;
typedef struct {
    int32_t kind;
    ref r;                 /* put target or condition */
    expr e;                /* put */
    int32_t b1, b2;        /* blocks (index of first statement, -1 = empty) */
    int32_t next;          /* next statement in its block */
} stmt;

typedef struct {
    const gen_tables *T;
    stream *r;
    stmt *st; int32_t nst, cap;
    int overflow;
} sampler;

static int32_t new_stmt(sampler *S) {
    if (S->nst == S->cap) { S->overflow = 1; return S->nst - 1; }
    memset(&S->st[S->nst], 0, sizeof(stmt));
    S->st[S->nst].b1 = S->st[S->nst].b2 = S->st[S->nst].next = -1;
    return S->nst++;
}

static ref get_ref(sampler *S) {                  /* ipt | scr | opt, then a digit */
    const uint32_t k = below(S->r, 30);
    const int32_t arrs[3] = {AR_IPT, AR_SCR, AR_OPT};
    ref x = {arrs[k / 10], (int32_t)(k % 10)};
    return x;
}

static ref put_ref(sampler *S) {                  /* scr | opt */
    const uint32_t k = below(S->r, 20);
    ref x = {k / 10 == 0 ? AR_SCR : AR_OPT, (int32_t)(k % 10)};
    return x;
}

static expr sample_expr(sampler *S, int32_t l) {
    expr e;
    memset(&e, 0, sizeof(e));
    if (l == 1) { e.kind = EX_CONST; e.c = (int32_t)below(S->r, 10); return e; }
    if (l == 4) { e.kind = EX_GET; e.g = get_ref(S); return e; }
    e.kind = EX_BIN;
    e.op = below(S->r, 2) == 0 ? '+' : '*';
    e.g = get_ref(S);
    if (l == 6) { e.rhs_const = 1; e.c = (int32_t)below(S->r, 10); }
    else { e.rhs_const = 0; e.h = get_ref(S); }
    return e;
}

static int32_t sample_block(sampler *S, int32_t l);

static int32_t sample_stmt(sampler *S, int32_t l) {
    const gen_tables *T = S->T;
    const uint32_t k = pick(S->r, T->s_off, T->s_cum, (uint32_t)l);
    const int32_t id = new_stmt(S);
    if (S->overflow) return id;
    if (T->s_kind[k] == 0) {
        S->st[id].kind = ST_PUT;
        S->st[id].r = put_ref(S);
        S->st[id].e = sample_expr(S, T->s_a[k]);
    } else if (T->s_kind[k] == 1) {
        S->st[id].kind = ST_IFE;
        S->st[id].r = get_ref(S);
        const int32_t b1 = sample_block(S, T->s_a[k]);
        const int32_t b2 = sample_block(S, T->s_b[k]);
        S->st[id].b1 = b1; S->st[id].b2 = b2;
    } else {
        S->st[id].kind = ST_WHL;
        S->st[id].r = get_ref(S);
        S->st[id].b1 = sample_block(S, T->s_a[k]);
    }
    return id;
}

static int32_t sample_block(sampler *S, int32_t l) {
    const gen_tables *T = S->T;
    int32_t first = -1, last = -1;
    for (;;) {
        const uint32_t k = pick(S->r, T->b_off, T->b_cum, (uint32_t)l);
        int32_t id;
        const int kind = T->b_kind[k];
        if (kind == 1) {
            id = new_stmt(S);
            if (!S->overflow) S->st[id].kind = ST_HLT;
        } else if (kind == 0) {
            id = sample_stmt(S, l);
        } else {
            id = sample_stmt(S, T->b_a[k]);
        }
        if (S->overflow) return first;
        if (first < 0) first = id; else S->st[last].next = id;
        last = id;
        if (kind != 2) return first;
        l = T->b_b[k];
    }
}

/* ---------------------------------------------------------------- lowering */
enum { LOD = 1, ADD = 2, MUL = 3, STO = 4, BNZ = 5, RD = 6, PRI = 7 };
enum { A_IMM = 0, A_ADDR = 1, A_NU = 2, A_LABEL = 3 };

typedef struct { int32_t op, kind, v1, v2; } insn;   /* A_ADDR: v1 region, v2 z; A_LABEL: v1 label */

typedef struct {
    insn *code; int32_t n, cap;
    int32_t *label; int32_t nlab, labcap;
    int32_t nout;
    int overflow;
} emitter;

static void emit(emitter *E, int32_t op, int32_t kind, int32_t v1, int32_t v2) {
    if (E->n == E->cap) { E->overflow = 1; return; }
    insn x = {op, kind, v1, v2};
    E->code[E->n++] = x;
}

static int32_t new_label(emitter *E) {
    if (E->nlab == E->labcap) { E->overflow = 1; return 0; }
    E->label[E->nlab] = -1;
    return E->nlab++;
}

static void mark(emitter *E, int32_t lab) { if (!E->overflow) E->label[lab] = E->n; }
static void jmp(emitter *E, int32_t lab) { emit(E, LOD, A_IMM, 1, 0); emit(E, BNZ, A_LABEL, lab, 0); }
static void get(emitter *E, ref g) { emit(E, LOD, A_IMM, 0, 0); emit(E, ADD, A_ADDR, g.arr, g.z); }

static void halt(emitter *E) {
    for (int32_t q = 0; q < E->nout; ++q) emit(E, PRI, A_ADDR, AR_OPT, q);
    emit(E, 0, A_IMM, 0, 0);
}

static void lower_block(emitter *E, const stmt *st, int32_t b) {
    for (; b >= 0; b = st[b].next) {
        const stmt *x = &st[b];
        if (x->kind == ST_HLT) {
            halt(E);
        } else if (x->kind == ST_PUT) {
            const expr *e = &x->e;
            if (e->kind == EX_CONST) emit(E, LOD, A_IMM, e->c, 0);
            else if (e->kind == EX_GET) get(E, e->g);
            else {
                get(E, e->g);
                emit(E, STO, A_NU, 0, 0);
                if (e->rhs_const) emit(E, LOD, A_IMM, e->c, 0);
                else get(E, e->h);
                emit(E, e->op == '+' ? ADD : MUL, A_NU, 0, 0);
            }
            emit(E, STO, A_ADDR, x->r.arr, x->r.z);
        } else if (x->kind == ST_IFE) {
            const int32_t lt = new_label(E), le = new_label(E);
            get(E, x->r);
            emit(E, BNZ, A_LABEL, lt, 0);
            lower_block(E, st, x->b2);
            jmp(E, le);
            mark(E, lt);
            lower_block(E, st, x->b1);
            mark(E, le);
        } else {
            const int32_t lh = new_label(E), lb = new_label(E), le = new_label(E);
            mark(E, lh);
            get(E, x->r);
            emit(E, BNZ, A_LABEL, lb, 0);
            jmp(E, le);
            mark(E, lb);
            lower_block(E, st, x->b1);
            jmp(E, lh);
            mark(E, le);
        }
    }
}

/* ---------------------------------------------------------------- entry */
/*
 * Programs first .. first+count-1 of the halting workload: words_out gets
 * each program's words back to back (at most n per program), prog_off the
 * offsets (count+1), tape_out / tape_off the input words (arity per program,
 * uniform w-bit words). out_arity 0 draws the output arity e uniformly
 * from 1..min(9, s); 1..min(9, s) fixes it (the draw is still taken, so the
 * body of program k does not depend on it). Returns 0, or -1 if a program could not be drawn
 * within the fixed working space (never for the grammar's lengths here) or
 * a parameter is out of range; *redraws counts programs redrawn because
 * their lowering did not fit n words.
 */
int gen_halting_programs(const gen_tables *T, uint64_t seed, uint64_t first, uint64_t count,
                         uint32_t ell, uint32_t s, uint32_t mu, uint32_t n, uint32_t w, int read_inputs,
                         uint32_t out_arity, int64_t *words_out, uint64_t *prog_off, int64_t *tape_out,
                         uint64_t *tape_off,
                         uint64_t *redraws) {
    if (T->L <= 15 || w < 1 || w > 64 || ell < 1 || s < 1) return -1;
    if (out_arity > (s < 9 ? s : 9)) return -1;
    enum { MAXST = 4096, MAXCODE = 8192, MAXLAB = 8192 };
    stmt *st = (stmt *)malloc(sizeof(stmt) * MAXST);
    insn *code = (insn *)malloc(sizeof(insn) * MAXCODE);
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * MAXLAB);
    if (!st || !code || !label) { free(st); free(code); free(label); return -1; }
    const uint64_t mask = w >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << w) - 1);
    const uint32_t in_max = ell < 9 ? ell : 9, out_max = s < 9 ? s : 9;
    uint64_t wo = 0, to = 0, nredraw = 0;
    int rc = 0;
    prog_off[0] = 0;
    tape_off[0] = 0;
    for (uint64_t k = 0; k < count && rc == 0; ++k) {
        const uint64_t pid = first + k;
        for (uint32_t attempt = 0;; ++attempt) {
            stream r = {seed, pid, 0x51A0000u + 4096u * attempt, 0, 0, {0, 0, 0, 0}, ~0u};
            const uint32_t nin = 1 + below(&r, in_max);
            const uint32_t drawn = 1 + below(&r, out_max);    /* drawn even when fixed: same body */
            const uint32_t nout = out_arity ? out_arity : drawn;
            sampler S = {T, &r, st, 0, MAXST, 0};
            const int32_t body = sample_block(&S, (int32_t)T->L - 15);
            emitter E = {code, 0, MAXCODE, label, 0, MAXLAB, (int32_t)nout, S.overflow};
            if (read_inputs)
                for (uint32_t z = 0; z < nin; ++z) emit(&E, RD, A_ADDR, AR_IPT, (int32_t)z);
            if (!E.overflow) lower_block(&E, st, body);
            halt(&E);
            if (E.overflow) { rc = -1; break; }
            const uint64_t m = (uint64_t)E.n, base = 2 * m;
            const uint64_t min_mem = base + 5 + ell + s + mu;
            if (min_mem > n) { nredraw++; continue; }
            const uint64_t region[3] = {base + 5, base + 5 + ell + s, base + 5 + ell};   /* ipt, scr, opt */
            const uint64_t size[3] = {nin, mu, nout};
            for (int32_t q = 0; q < E.n; ++q) {
                const insn *x = &code[q];
                uint64_t arg = 0;
                if (x->kind == A_IMM) arg = (uint64_t)(int64_t)x->v1;
                else if (x->kind == A_NU) arg = base;
                else if (x->kind == A_ADDR) arg = region[x->v1] + (uint64_t)x->v2 % size[x->v1];
                else arg = 2 * (uint64_t)label[x->v1];
                words_out[wo++] = x->op;
                words_out[wo++] = (int64_t)arg;
            }
            prog_off[k + 1] = wo;
            for (uint32_t z = 0; z < nin; ++z) {
                const uint64_t lo = draw(seed, 0x51B0000u, pid, z);
                const uint64_t hi = w > 32 ? draw(seed, 0x51C0000u, pid, z) : 0;
                tape_out[to++] = (int64_t)(((hi << 32) | lo) & mask);
            }
            tape_off[k + 1] = to;
            break;
        }
    }
    free(st); free(code); free(label);
    *redraws = nredraw;
    return rc;
}
