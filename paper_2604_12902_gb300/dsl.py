"""Heapless array language and its lowering to word-RASP programs (Sec. 2.2).

Grammar (Sec. 2.2):

    F ::= fun f0 ( ipt : W ^ N ) -> W ^ N { B }      N ::= 1 .. 9
    B ::= S | S ; B | hlt                             Z ::= 0 | N
    S ::= P = E | ife G { B } { B } | whl G { B }
    G ::= ipt [ Z ] | scr [ Z ] | opt [ Z ]           P ::= scr [ Z ] | opt [ Z ]
    E ::= G + G | G * G | G + Z | G * Z | G | Z

Lowering rules (Sec. 2.2, "Fun", "Get", "Put", (+), (x), "Ife", "While",
"Seq", "Halt"), written as instruction sequences:

    Get   a[z]          ->  LOD 0 ; ADD [[a]]_z
    Z     z             ->  LOD z                       (a constant leaves z in a)
    Put   a[z] = E      ->  <E> ; STO [[a]]_z
    I1 + I2             ->  <I1> ; STO nu ; <I2> ; ADD nu     (MUL for *)
    ife I {B1} {B2}     ->  <I> ; BNZ lt ; <B2> ; JMP le ; lt: <B1> ; le:
    whl I {B}           ->  lh: <I> ; BNZ lb ; JMP le ; lb: <B> ; JMP lh ; le:
    hlt, end of f0      ->  PRI q_0 .. PRI q_(e-1) ; HLT
    JMP l               ->  LOD 1 ; BNZ l            HLT -> the invalid pair 0 0

Memory regions (Sec. 2.2): after the 2m program words come the reserved
word nu and four more reserved words, then ipt (l words), opt (s words) and
scr (mu words), so 5 + l + s + mu + 2m <= n, and
[[a]]_z = M[2m + [[a]] + (z mod |a|)] with |ipt| = N (declared input arity),
|opt| = e (declared output arity) and |scr| = mu.

The Fun rule reads no input: the ipt region starts as zeros, as in the
busy-beaver runs of App. B. ``read_inputs=True`` prepends one ``RD`` per
input word so that a program can consume its tape x; it changes tau_h by N.
"""
from __future__ import annotations

import re
from dataclasses import dataclass

LOD, ADD, MUL, STO, BNZ, RD, PRI = 1, 2, 3, 4, 5, 6, 7
RESERVED = 5          # nu plus four more reserved words before the arrays


# ------------------------------------------------------------------ parsing
_TOKEN = re.compile(r"\s*(->|[A-Za-z_][A-Za-z_0-9]*|\d+|[()\[\]{}:;^=+*])")


def tokenize(src: str):
    pos, out = 0, []
    src = src.strip()
    while pos < len(src):
        m = _TOKEN.match(src, pos)
        if not m:
            raise SyntaxError("bad character at %d: %r" % (pos, src[pos:pos + 10]))
        out.append(m.group(1))
        pos = m.end()
        while pos < len(src) and src[pos].isspace():
            pos += 1
    return out


@dataclass
class Fun:
    arity: int        # N of ipt
    out_arity: int    # e
    body: list        # block


class _Parser:
    def __init__(self, toks):
        self.t, self.k = toks, 0

    def peek(self, off=0):
        return self.t[self.k + off] if self.k + off < len(self.t) else None

    def eat(self, want=None):
        tok = self.peek()
        if tok is None or (want is not None and tok != want):
            raise SyntaxError("expected %r, got %r at token %d" % (want, tok, self.k))
        self.k += 1
        return tok

    def digit(self, lo):
        tok = self.eat()
        if not tok.isdigit() or not (lo <= int(tok) <= 9):
            raise SyntaxError("expected a digit in %d..9, got %r" % (lo, tok))
        return int(tok)

    def fun(self) -> Fun:
        self.eat("fun"); self.eat("f0"); self.eat("(")
        self.eat("ipt"); self.eat(":"); self.eat("W"); self.eat("^")
        n_in = self.digit(1)
        self.eat(")"); self.eat("->"); self.eat("W"); self.eat("^")
        n_out = self.digit(1)
        self.eat("{")
        body = self.block()
        self.eat("}")
        if self.peek() is not None:
            raise SyntaxError("trailing tokens after f0")
        return Fun(n_in, n_out, body)

    def block(self):
        if self.peek() == "hlt":
            self.eat()
            return [("hlt",)]
        stmts = [self.stmt()]
        while self.peek() == ";":
            self.eat()
            if self.peek() == "hlt":
                self.eat()
                stmts.append(("hlt",))
                break
            stmts.append(self.stmt())
        return stmts

    def ref(self, allowed):
        name = self.eat()
        if name not in allowed:
            raise SyntaxError("expected one of %s, got %r" % (allowed, name))
        self.eat("[")
        z = self.digit(0)
        self.eat("]")
        return (name, z)

    def stmt(self):
        tok = self.peek()
        if tok == "ife":
            self.eat()
            g = self.ref(("ipt", "scr", "opt"))
            self.eat("{"); b1 = self.block(); self.eat("}")
            self.eat("{"); b2 = self.block(); self.eat("}")
            return ("ife", g, b1, b2)
        if tok == "whl":
            self.eat()
            g = self.ref(("ipt", "scr", "opt"))
            self.eat("{"); b = self.block(); self.eat("}")
            return ("whl", g, b)
        p = self.ref(("scr", "opt"))
        self.eat("=")
        return ("put", p, self.expr())

    def expr(self):
        if self.peek() is not None and self.peek().isdigit():
            return ("const", self.digit(0))
        g = self.ref(("ipt", "scr", "opt"))
        if self.peek() in ("+", "*"):
            op = self.eat()
            if self.peek() is not None and self.peek().isdigit():
                rhs = ("const", self.digit(0))
            else:
                rhs = ("get", self.ref(("ipt", "scr", "opt")))
            return ("bin", op, ("get", g), rhs)
        return ("get", g)


def parse(src: str) -> Fun:
    return _Parser(tokenize(src)).fun()


# ----------------------------------------------------------------- lowering
@dataclass
class Lowered:
    words: list          # program words (2m of them), Python ints (may be negative)
    m: int               # instructions
    layout: dict         # region -> absolute base address, and 'nu'
    sizes: dict          # region -> length
    min_mem: int         # smallest legal n

    def address(self, region: str, z: int) -> int:
        return self.layout[region] + (z % self.sizes[region])


class _Emitter:
    def __init__(self, out_arity):
        self.code = []       # [op, operand] with operand int | ('addr', r, z) | ('nu',) | ('label', id)
        self.labels = {}
        self.nlab = 0
        self.e = out_arity

    def new_label(self):
        self.nlab += 1
        return self.nlab

    def mark(self, lab):
        self.labels[lab] = len(self.code)

    def emit(self, op, arg):
        self.code.append((op, arg))

    def jmp(self, lab):
        self.emit(LOD, 1)
        self.emit(BNZ, ("label", lab))

    def get(self, ref):
        self.emit(LOD, 0)
        self.emit(ADD, ("addr",) + ref)

    def value(self, e):
        if e[0] == "const":
            self.emit(LOD, e[1])
        elif e[0] == "get":
            self.get(e[1])
        else:
            _, op, lhs, rhs = e
            self.value(lhs)
            self.emit(STO, ("nu",))
            self.value(rhs)
            self.emit(ADD if op == "+" else MUL, ("nu",))

    def halt(self):
        for q in range(self.e):
            self.emit(PRI, ("addr", "opt", q))
        self.emit(0, 0)

    def block(self, stmts):
        for st in stmts:
            kind = st[0]
            if kind == "hlt":
                self.halt()
            elif kind == "put":
                self.value(st[2])
                self.emit(STO, ("addr",) + st[1])
            elif kind == "ife":
                lt, le = self.new_label(), self.new_label()
                self.get(st[1])
                self.emit(BNZ, ("label", lt))
                self.block(st[3])
                self.jmp(le)
                self.mark(lt)
                self.block(st[2])
                self.mark(le)
            elif kind == "whl":
                lh, lb, le = self.new_label(), self.new_label(), self.new_label()
                self.mark(lh)
                self.get(st[1])
                self.emit(BNZ, ("label", lb))
                self.jmp(le)
                self.mark(lb)
                self.block(st[2])
                self.jmp(lh)
                self.mark(le)
            else:
                raise ValueError(kind)


def lower(src_or_fun, ell: int = 10, s: int = 2, mu: int = 10,
          read_inputs: bool = False) -> Lowered:
    """Lower a program of the array language to RASP words (Sec. 2.2)."""
    f = parse(src_or_fun) if isinstance(src_or_fun, str) else src_or_fun
    if f.arity > ell or f.out_arity > s:
        raise ValueError("ipt/opt do not fit the tapes (N <= l, e <= s)")
    em = _Emitter(f.out_arity)
    if read_inputs:
        for z in range(f.arity):
            em.emit(RD, ("addr", "ipt", z))
    em.block(f.body)
    em.halt()                                  # Fun: C ; PRI q_i ; HLT
    m = len(em.code)
    base = 2 * m
    layout = {"nu": base, "ipt": base + RESERVED, "opt": base + RESERVED + ell,
              "scr": base + RESERVED + ell + s}
    sizes = {"ipt": f.arity, "opt": f.out_arity, "scr": mu}
    words = []
    for op, arg in em.code:
        if isinstance(arg, tuple):
            if arg[0] == "nu":
                arg = layout["nu"]
            elif arg[0] == "addr":
                arg = layout[arg[1]] + (arg[2] % sizes[arg[1]])
            elif arg[0] == "label":
                arg = 2 * em.labels[arg[1]]
        words += [op, arg]
    return Lowered(words, m, layout, sizes, base + RESERVED + ell + s + mu)
