"""Build-time generator of the per-process amplitude code for g g -> t tbar + n g.

The paper's amplitudes are generated per process by a meta-program that
emits HELAS-style call chains (Sec. 3.1); this is the library's own, much
smaller generator for the processes it ships.  For n gluons on the top line it

  * counts the tree-level Feynman diagrams (3, 16, 123 for n = 2, 3, 4) from
    the 3-gluon, 4-gluon and quark-gluon vertices;
  * derives the colour matrix C_{sigma tau} = sum_colours
    (t^sigma)^*_{ij} (t^tau)_{ij} of the colour-ordered basis
    (t^{a_sigma1} ... t^{a_sigman})_{ij} exactly, by Fierz reduction of
    SU(N) traces in rational arithmetic at N = 3;
  * emits a CUDA device function that evaluates every colour-ordered
    amplitude as chains of vertex and propagator calls -- off-shell gluon
    currents (3- and 4-gluon vertices), off-shell top currents (quark-gluon
    vertex + top propagator) emitted depth-first over the orderings'
    suffixes, the amputated spinor of each ordering closed at once with the
    top's ubar of both helicities -- sharing every
    sub-current between the n! orderings (the sum over all Feynman diagrams,
    organised so that no diagram's chain is recomputed), with the helicity
    sum written as nested loops over the external helicities and every
    gluon current computed at the outermost loop level on which it depends;
  * shares, between the two orderings in which it occurs, every slash of a
    multi-gluon current on a top spinor (reflection identity), hoists the
    antitop current of the fixed-helicity gluon out of the inner loops, and
    sums colours in pair form with one FMA accumulator per distinct entry;
  * counts the floating-point operations of the emitted code.

Couplings are stripped (g = 1): every partial amplitude carries exactly g^n,
restored as (4 pi alpha_s)^n on |M|^2.

Run ``python -m paper_2312_07440_gb300.gen.qcd_gen`` to regenerate
``csrc/gen_qcd_*.cuh`` (the generated headers are committed).
"""
from __future__ import annotations

import itertools
import math
import os
from fractions import Fraction

# ---------------------------------------------------------------------------
# colour algebra: Fierz reduction of traces of SU(N) generators
# ---------------------------------------------------------------------------
NC = 3


def _reduce(coef, traces):
    """Fully contract a product of traces of generator words.

    traces: tuple of tuples of adjoint labels; each label occurs exactly twice
    over the whole product.  Uses, with T = t^a summed over a,
      Tr(X t^a Y t^a) = 1/2 Tr(X) Tr(Y) - 1/(2N) Tr(X Y)
      Tr(X t^a) Tr(Y t^a) = 1/2 Tr(X Y) - 1/(2N) Tr(X) Tr(Y)
    and Tr(1) = N.  Returns an exact Fraction.
    """
    # find a label
    for ti, tr in enumerate(traces):
        if tr:
            lab = tr[0]
            break
    else:
        return coef * Fraction(NC) ** len(traces)
    pos = [(ti, k) for ti, tr in enumerate(traces) for k, x in enumerate(tr) if x == lab]
    assert len(pos) == 2
    (t1, k1), (t2, k2) = pos
    rest = [tr for ti, tr in enumerate(traces) if ti not in (t1, t2)]
    half = Fraction(1, 2)
    inv2n = Fraction(1, 2 * NC)
    if t1 == t2:
        tr = traces[t1]
        # rotate so that the first occurrence is at position 0: Tr(t^a Y t^a X)
        rot = tr[k1:] + tr[:k1]
        j = rot.index(lab, 1)
        Y, X = rot[1:j], rot[j + 1:]
        return (_reduce(coef * half, tuple(rest) + (X, Y)) - _reduce(coef * inv2n, tuple(rest) + (X + Y,)))
    a, b = traces[t1], traces[t2]
    X = a[k1 + 1:] + a[:k1]  # Tr(t^a X) with X cyclically after a
    Y = b[k2 + 1:] + b[:k2]
    return (_reduce(coef * half, tuple(rest) + (X + Y,)) - _reduce(coef * inv2n, tuple(rest) + (X, Y)))


def orderings(n):
    return list(itertools.permutations(range(n)))


def colour_matrix(n):
    """C[s][t] = Tr(t^{sigma_n} ... t^{sigma_1} t^{tau_1} ... t^{tau_n}) summed
    over the adjoint labels, as exact Fractions (lexicographic orderings)."""
    perms = orderings(n)
    C = []
    for s in perms:
        row = []
        for t in perms:
            word = tuple(reversed(s)) + tuple(t)
            row.append(_reduce(Fraction(1), (word,)))
        C.append(row)
    return C


def colour_matrix_int(n):
    """(integer matrix, common denominator) with C = Cint / den."""
    C = colour_matrix(n)
    den = 1
    for row in C:
        for x in row:
            den = den * x.denominator // math.gcd(den, x.denominator)
    return [[int(x * den) for x in row] for row in C], den


def colour_pairs(Cint):
    """Pair form of sum_ij Cint_ij Re(A_i^* A_j): [(i, j, c)] over i <= j with
    Cint_ij != 0, c = Cint_ii on the diagonal and 2 Cint_ij off it."""
    K = len(Cint)
    return [(i, j, Cint[i][j] * (1 if i == j else 2)) for i in range(K) for j in range(i, K) if Cint[i][j]]


def colour_rows(Cint):
    """Row form of 2 sum_ij Cint_ij Re(A_i^* A_j) (the factor 2 of the helicity
    flip folded in): [(i, [(j, coefficient)])], z_i = 2 Cint_ii A_i + 4 sum_{j>i}
    Cint_ij A_j, and the sum is sum_i Re(A_i^* z_i)."""
    K = len(Cint)
    return [(i, [(i, 2 * Cint[i][i])] + [(j, 4 * Cint[i][j]) for j in range(i + 1, K) if Cint[i][j]])
            for i in range(K)]


# ---------------------------------------------------------------------------
# diagram counting (unordered, colour-dressed Feynman graphs)
# ---------------------------------------------------------------------------
def _set_partitions(items, k):
    """Unordered partitions of the tuple ``items`` into k nonempty blocks."""
    items = list(items)
    if k == 1:
        yield (tuple(items),)
        return
    first, rest = items[0], items[1:]
    # block containing `first`
    for r in range(0, len(rest) + 1):
        for others in itertools.combinations(rest, r):
            block = (first,) + others
            remaining = tuple(x for x in rest if x not in others)
            if len(remaining) < k - 1:
                continue
            for sub in _set_partitions(remaining, k - 1):
                yield (block,) + sub


def diagram_count(n):
    """Number of tree diagrams for t tbar + n gluons (3g, 4g, qqg vertices)."""
    from functools import lru_cache

    @lru_cache(None)
    def dg(S):
        if len(S) == 1:
            return 1
        tot = 0
        for a, b in _set_partitions(S, 2):
            tot += dg(a) * dg(b)
        if len(S) >= 3:
            for a, b, c in _set_partitions(S, 3):
                tot += dg(a) * dg(b) * dg(c)
        return tot

    @lru_cache(None)
    def df(S):
        if not S:
            return 1
        tot = 0
        for r in range(1, len(S) + 1):
            for sub in itertools.combinations(S, r):
                rest = tuple(x for x in S if x not in sub)
                tot += dg(sub) * df(rest)
        return tot

    return df(tuple(range(n)))


# ---------------------------------------------------------------------------
# code emission
# ---------------------------------------------------------------------------
# floating-point operations of the device primitives in helas.cuh (real
# operations; an FMA counts 2).  Kept in step with helas.cuh by hand.
PAIRS_MAX_K = 6  # colour sums of up to this many orderings by pairs (see emit_process)
ROW_ACCS = 4     # accumulators per top helicity for the row-wise colour sum

FLOPS = {
    "vvv": 156,      # 3-gluon vertex with folded propagator factor
    "vvvv_acc": 193, # 4-gluon vertex accumulated
    "slash": 64,     # Jslash psi from the vector J
    "slash_w": 56,   # Jslash psi from J's Weyl-block form
    "weyl": 8,       # Weyl-block form of a vector
    "sp_add": 8,     # spinor accumulate
    "fprop": 58,     # c (qslash + m) chi
    "fcur": 72,      # ubar gamma^mu psi
    "dot": 30,       # complex Minkowski product
    "rowcol": 30,    # ubar . X (row times column spinor)
    "cadd": 2,
}


def seq_name(prefix, seq):
    return prefix + "_".join(str(x) for x in seq) if seq else prefix + "E"


def mask(seq):
    m = 0
    for x in seq:
        m |= 1 << x
    return m


class Emitter:
    def __init__(self, n):
        self.n = n
        self.flops_per_level = [0] * (n + 2)  # flops emitted at each loop level

    def count(self, level, key, times=1):
        self.flops_per_level[level] += FLOPS[key] * times


def emit_process(name, n, outgoing_gluons, n_identical, hoist_weyl=True, share_fp32=0):
    """Emit the helicity-summed, couplings-stripped colour sum for t tbar + n g.

    Loop levels 0..n-1: gluon helicities; level n: antitop (the top helicity is
    summed inside it: both amplitudes of every ordering are formed at once).
    Level 0 is fixed (helicity-flip symmetry); the returned device function
    sums over the helicities of one lane, levels 1..LB taking their helicity
    bits from the lane index.

    hoist_weyl: form each polarisation's Weyl-block form once per level trip
    and both antitop variants of S(0) once per helicity sum (fewer operations,
    more live registers; it pays where the state is small).
    """
    em = Emitter(n)
    perms = orderings(n)
    K = len(perms)
    Cint, den = colour_matrix_int(n)
    lines = []
    w = lines.append
    w(f"// ---- generated by gen/qcd_gen.py: {name} (g g -> t tbar + {n - 2} g), do not edit ----")
    w(f"// {diagram_count(n)} Feynman diagrams, {K} colour orderings, {2 ** (n + 2)} helicities.")
    w(f"// colour matrix C = Cint / {den}")
    w("#pragma once")
    w('#include "colour_mma.cuh"')
    w('#include "qcd.cuh"')
    w("")
    w(f"namespace rw {{ namespace {name} {{")
    w(f"constexpr int NG = {n};")
    w(f"constexpr int NEXT = {n + 2};")
    w(f"constexpr int K = {K};")
    w(f"constexpr int NHEL = {2 ** (n + 2)};")
    w(f"constexpr int NDIAG = {diagram_count(n)};")
    w(f"constexpr int MAX_LB = {n};  // helicity levels that can be spread over lanes")
    njs = sum(math.perm(n, L) // 2 for L in range(3, n + 1))
    w(f"constexpr int NJS = {njs};  // currents of 3+ gluons, one JStore slot each")
    w(f"constexpr int CDEN = {den};")
    w(f"constexpr int IDENT = {n_identical};  // identical outgoing gluons (1/IDENT!)")
    w(f"constexpr unsigned OUTGOING_GLUONS = {sum(1 << g for g in outgoing_gluons)}u;  // bit g: gluon g outgoing")
    flat = ", ".join(str(x) for row in Cint for x in row)
    w(f"__host__ __device__ constexpr int cint(int i, int j) {{ constexpr int c[K * K] = {{{flat}}}; return c[i * K + j]; }}")
    w(f"constexpr int ORDER[K][NG] = {{{', '.join('{' + ', '.join(map(str, p)) + '}' for p in perms)}}};")
    w(f"static __device__ const short CI[K * K] = {{{flat}}};  // row-major C_int for the tensor-core sum")
    w("")
    w("// Sum over this lane's helicities of sum_{s,t} Cint_st Re(A_s^* A_t), g = 1;")
    w("// helicities with gluon 0 at +1 only, doubled (J^dagger C J(h) = J^dagger C J(-h)).")
    w("// CM: colour sum by FMA (CM_FMA, any R) or on the tensor cores (CM_FP16/CM_BF16, R = float);")
    w("// CM_STORE_FP16/CM_STORE_BF16: no colour sum here, each J vector goes to sink->put()")
    w("// for a later tensor-core pass (the return value is then 0).")
    w("template <class R, int LB, int CM = CM_FMA, bool JS = false, class Sink = NoSink>")
    w("__device__ __forceinline__ R hel_sum(const QcdExt<R, NG>& X, const QcdKin<R, NG>& Kn, int lane,")
    w("                                     [[maybe_unused]] Sink* sink = nullptr) {")
    w("  static_assert(CM == CM_FMA || sizeof(R) == 4, \"tensor-core colour sum takes FP32 amplitudes\");")
    w("  constexpr bool MMA = CM == CM_FP16 || CM == CM_BF16;")
    w("  const ColourMma<K, MMA ? CM : CM_FP16> cmma(MMA ? CI : nullptr, JS ? NJS * 32 : 0);")
    w("  JStore<R, NJS, JS> js;")
    w("  R acc = R(0);")
    # Colour sum by FMA.  Up to PAIRS_MAX_K orderings: sum over the pairs
    # i <= j with C_ij != 0 of c_ij Re(A_i^* A_j) (c_ii = C_ii, c_ij = 2 C_ij),
    # each product accumulated by two FMAs into one accumulator per distinct
    # c and top helicity (two independent chains), scaled once after the loops.  Larger K: z = C A row by row, then
    # Re(A_i^* z_i) into acc (C's symmetric half, coefficients pre-scaled).
    pairs = K <= PAIRS_MAX_K
    coef = {}
    if pairs:
        for _, _, c in colour_pairs(Cint):
            coef.setdefault(c, len(coef))
        ccs = [f"cc{k}_{h} = R(0)" for h in (0, 1) for k in range(len(coef))]
        w(f"  [[maybe_unused]] R {', '.join(ccs)};  // per distinct c_ij and top helicity")
    else:
        # rows spread over ROW_ACCS accumulators per top helicity: short FMA
        # dependency chains
        czs = [f"cz{h}_{k} = R(0)" for h in (0, 1) for k in range(ROW_ACCS)]
        w(f"  [[maybe_unused]] R {', '.join(czs)};")
    ind = "  "

    def jref(sq):
        """Expression for the current of the gluon sequence sq."""
        if len(sq) == 1:
            return f"E{sq[0]}"
        if sq in slot:
            return f"js.get({slot[sq]})"
        if sq in alias:
            return alias[sq]
        return seq_name("J", sq)

    # all sequences of distinct gluons, by length
    seqs = {L: list(itertools.permutations(range(n), L)) for L in range(1, n + 1)}
    canon = {}  # J name for reversed sequences
    nlev = n + 1

    def open_level(L, hvar, sel):
        nonlocal ind
        if L == 0:
            # helicity-flip symmetry: J^dagger C J is the same for h and -h
            # (tree-level QCD with real momenta), so gluon 0 keeps helicity +
            # and the sum is doubled.
            w(f"{ind}{{")
            ind += "  "
            w(f"{ind}const int {hvar} = 0;")
            w(f"{ind}{sel}")
            return
        bit = f"((lane >> (LB - {L})) & 1)"
        w(f"{ind}#pragma unroll 1")
        w(f"{ind}for (int i{L} = 0; i{L} < (LB >= {L} ? 1 : 2); ++i{L}) {{")
        ind += "  "
        w(f"{ind}const int {hvar} = LB >= {L} ? {bit} : i{L};")
        w(f"{ind}{sel}")

    # gluon levels.  Currents of three or more gluons live in a JStore slot
    # (registers, or this thread's slice of shared memory when JS is set):
    # they are written once and read back at every use, so the compiler need
    # not keep all of them in registers through the antitop level.
    slot = {}    # canonical sequence -> slot
    wform = {}   # canonical sequence -> name of its Weyl form
    alias = {}   # any sequence -> expression
    for g in range(n):
        open_level(g, f"h{g}", f"const cv<R> E{g} = h{g} ? X.eps[{g}][1] : X.eps[{g}][0];")
        if hoist_weyl:
            w(f"{ind}const ws<R> W{g} = weyl_form(E{g});")
            em.count(g, "weyl")
        if g == 0 and hoist_weyl:
            # S(0) depends on the antitop helicity and on gluon 0's, which is
            # fixed: both antitop variants are formed here once instead of at
            # every trip of the inner loops (unless the antitop helicity is a
            # lane bit, when each lane forms its own below).
            w(f"{ind}[[maybe_unused]] sp<R> S_0v0, S_0v1;")
            w(f"{ind}if constexpr (LB < {n}) {{")
            w(f"{ind}  S_0v0 = fprop(Kn.qc[1], Kn.mc[1], slash(W0, X.v[0]));")
            w(f"{ind}  S_0v1 = fprop(Kn.qc[1], Kn.mc[1], slash(W0, X.v[1]));")
            w(f"{ind}}}")
            em.count(0, "slash_w", 2)
            em.count(0, "fprop", 2)
        for L in range(2, n + 1):
            for sq in seqs[L]:
                if max(sq) != g:
                    continue
                nm = seq_name("J", sq)
                rv = tuple(reversed(sq))
                if rv in canon:
                    # reflection identity J(reversed) = (-1)^{L+1} J
                    src = jref(rv)
                    expr = f"neg({src})" if L % 2 == 0 else src
                    if rv in slot:
                        alias[sq] = expr
                    else:
                        w(f"{ind}const cv<R> {nm} = {expr};")
                    continue
                canon[sq] = nm
                m = mask(sq)
                terms = []
                for c in range(1, L):
                    a, b = sq[:c], sq[c:]
                    terms.append(f"{jref(a)}, Kn.P[{mask(a)}], {jref(b)}, Kn.P[{mask(b)}], Kn.cg[{m}]")
                    em.count(g, "vvv")
                w(f"{ind}cv<R> {nm} = vvv({terms[0]});")
                for t in terms[1:]:
                    w(f"{ind}vvv_acc({nm}, {t});")  # fused accumulation
                    em.count(g, "cadd", 8)
                for c in range(1, L):
                    for d in range(c + 1, L):
                        a, b, cc = sq[:c], sq[c:d], sq[d:]
                        w(f"{ind}vvvv_acc({nm}, {jref(a)}, {jref(b)}, {jref(cc)}, Kn.c4[{m}]);")
                        em.count(g, "vvvv_acc")
                if L >= 3:
                    slot[sq] = len(slot)
                    w(f"{ind}js.put({slot[sq]}, {nm});")
                elif L == n and hoist_weyl:
                    # a full-length current is only ever slashed: keep its Weyl form
                    wform[sq] = f"W{nm}"
                    w(f"{ind}const ws<R> W{nm} = weyl_form({nm});")
                    em.count(g, "weyl")
    # antitop level: the fermion currents psi(rho) = S_rho (rho a proper
    # sequence of gluons attached from the antitop end), the amputated spinor
    # X(sigma) = sum_c Jslash(sigma[..c]) psi(sigma[c+1..]) of every ordering and
    # its amplitudes A(sigma, h_t) = ubar(h_t) X(sigma) for both top helicities
    # (the top level is folded in: X dies as soon as it is closed).  The
    # spinors are emitted depth-first over the suffix tree -- S(d), S(c d),
    # S(b c d), then X(a b c d) -- so only the current path of spinors is live
    # at any time.
    open_level(n, f"h{n}", f"const sp<R> S_E = h{n} ? X.v[1] : X.v[0];")

    def jn(sq):
        return f"W{sq[0]}" if len(sq) == 1 and hoist_weyl else jref(sq)

    def slash_kind(sq):
        return "slash_w" if len(sq) == 1 and hoist_weyl else "slash"

    # Every term Jslash(a) psi(b) with |a| >= 2 occurs twice at this level:
    # in the node a+b and in rev(a)+b, where J(rev a) = (-1)^{|a|+1} J(a).
    # The second occurrence reuses the first's spinor Y (one slash instead of
    # two) in FP64, where a slash costs far more than keeping Y in registers
    # or L1; in FP32 only when the two uses are at most share_fp32 statements
    # apart (a distant Y would spill and cost more than the slash it saves).
    # A node starts from its shared spinors (+-Y, no products) and takes its
    # single-gluon term last as a fused slash-accumulate.
    ops = []  # ("line", text) or ("node", target, declaration, [(a, b) terms], single-gluon term)

    def visit(suffix):
        rest = [g for g in range(n) if g not in suffix]
        if len(rest) == 1:
            sg = (rest[0],) + suffix
            k = perms.index(sg)
            ops.append(("node", f"X{k}", f"sp<R> X{k}", [(sg[:c], sg[c:]) for c in range(2, n + 1)], (sg[:1], sg[1:])))
            ops.append(("line", f"const cx<R> A{k}_0 = rowcol(X.ub[0], X{k}), A{k}_1 = rowcol(X.ub[1], X{k});"))
            em.count(n, "rowcol", 2)
            return
        for b0 in rest:
            rho = (b0,) + suffix
            nm = seq_name("S_", rho)
            if rho == (0,) and hoist_weyl:
                ops.append(("line", "sp<R> S_0;"))
                ops.append(("line", f"if constexpr (LB < {n}) S_0 = h{n} ? S_0v1 : S_0v0;"))
                ops.append(("line", "else S_0 = fprop(Kn.qc[1], Kn.mc[1], slash(W0, S_E));"))
                visit(rho)
                continue
            ops.append(("node", f"t{nm}", f"sp<R> t{nm}", [(rho[:c], rho[c:]) for c in range(2, len(rho) + 1)],
                        (rho[:1], rho[1:])))
            ops.append(("line", f"const sp<R> {nm} = fprop(Kn.qc[{mask(rho)}], Kn.mc[{mask(rho)}], t{nm});"))
            em.count(n, "fprop")
            visit(rho)
    visit(())

    def share_key(a, b):
        ca = a if a in canon else tuple(reversed(a))
        sgn = 1 if ca == a or len(a) % 2 == 1 else -1
        return (ca, b), sgn

    uses = {}
    for i, op in enumerate(ops):
        if op[0] == "node":
            for a, b in op[3]:
                uses.setdefault(share_key(a, b)[0], []).append(i)
    assert all(len(u) == 2 for u in uses.values())
    share_gaps = sorted(u[1] - u[0] for u in uses.values())
    w(f"{ind}constexpr bool SH = sizeof(R) == 8;  // share every repeated slash (FP64)")
    for i, op in enumerate(ops):
        if op[0] == "line":
            w(f"{ind}{op[1]}")
            continue
        _, tgt, decl, terms, (a1, b1) = op
        w1 = f"{jn(a1)}, {seq_name('S_', b1)}"
        em.count(n, slash_kind(a1))
        if not terms:
            w(f"{ind}{decl} = slash({w1});")
            continue
        w(f"{ind}{decl};")
        info = []
        for t, (a, b) in enumerate(terms):
            key, sgn = share_key(a, b)
            first, second = uses[key]
            yn = "Y" + "_".join(map(str, key[0])) + "__" + seq_name("S_", b)[2:]
            near = second - first <= share_fp32
            info.append((a, b, key, sgn, i == first, yn, near))
            if i == first:
                w(f"{ind}[[maybe_unused]] sp<R> {yn};  // Jslash({','.join(map(str, key[0]))}) psi({seq_name('S_', b)[2:]})")
                em.count(n, "slash_w" if key[0] in wform else "slash")
            if t > 0:
                em.count(n, "sp_add")
        em.count(n, "sp_add")  # the single-gluon term, accumulated

        def shared_form(ind2, conds):
            for t, ((a, b, key, sgn, first, yn, near), cond) in enumerate(zip(info, conds)):
                sb = seq_name("S_", b)
                if first:
                    w(f"{ind2}if constexpr ({cond}) {yn} = slash({wform.get(key[0], jref(key[0]))}, {sb});")
                if t == 0:
                    ys = yn if sgn > 0 else f"spneg({yn})"
                    w(f"{ind2}if constexpr ({cond}) {tgt} = {ys}; else {tgt} = slash({jref(a)}, {sb});")
                else:
                    w(f"{ind2}if constexpr ({cond}) {'spadd' if sgn > 0 else 'spsub'}({tgt}, {yn}); "
                      f"else slash_acc({tgt}, {jref(a)}, {sb});")
            w(f"{ind2}slash_acc({tgt}, {w1});  // single-gluon term, fused")

        if any(x[6] for x in info):
            shared_form(ind, ["true" if x[6] else "SH" for x in info])
        else:
            # nothing shared in FP32: there the single-gluon term goes first, as
            # the node's chain starts from the spinor just computed
            w(f"{ind}if constexpr (SH) {{")
            shared_form(ind + "  ", ["true"] * len(info))
            w(f"{ind}}} else {{")
            w(f"{ind}  {tgt} = slash({w1});")
            for a, b, *_ in info:
                w(f"{ind}  slash_acc({tgt}, {jref(a)}, {seq_name('S_', b)});")
            w(f"{ind}}}")
    # colour sums of both top helicities
    w(f"{ind}if constexpr (CM != CM_FMA) {{")
    for h in (0, 1):
        w(f"{ind}  const cx<float> Aa{h}[K] = {{{', '.join(f'A{k}_{h}' for k in range(K))}}};")
    w(f"{ind}  if constexpr (MMA) {{")
    w(f"{ind}    acc += R(2) * (cmma.sum(Aa0) + cmma.sum(Aa1));  // x2 helicity flip")
    w(f"{ind}  }} else {{")
    w(f"{ind}    sink->put(Aa0);")
    w(f"{ind}    sink->put(Aa1);")
    w(f"{ind}  }}")
    w(f"{ind}}} else {{")
    ind += "  "
    if pairs:
        for h in (0, 1):
            for i, j, c in colour_pairs(Cint):
                k = coef[c]
                a, b = f"A{i}_{h}", f"A{j}_{h}"
                w(f"{ind}cc{k}_{h} = fmadd({a}.r, {b}.r, fmadd({a}.i, {b}.i, cc{k}_{h}));")
                em.flops_per_level[n] += 4
    else:
        # symmetric half, x2 symmetric colour sum, x2 helicity flip folded in:
        # acc += Re(A_i^* (2 C_ii A_i + 4 sum_{j>i} C_ij A_j))
        for h in (0, 1):
            for i, row in colour_rows(Cint):
                parts_r = [f"R({cf}) * A{j}_{h}.r" for j, cf in row]
                parts_i = [f"R({cf}) * A{j}_{h}.i" for j, cf in row]
                w(f"{ind}{{ const R zr = {' + '.join(parts_r)}; const R zi = {' + '.join(parts_i)};")
                k = f"cz{h}_{i % ROW_ACCS}"
                w(f"{ind}  {k} = fmadd(A{i}_{h}.r, zr, fmadd(A{i}_{h}.i, zi, {k})); }}")
                em.flops_per_level[n] += 4 * len(parts_r) + 4
    ind = ind[:-2]
    w(f"{ind}}}")
    for L in range(nlev - 1, -1, -1):
        ind = ind[:-2]
        w(f"{ind}}}")
    if pairs:
        combo = " + ".join(f"R({c}) * (cc{k}_0 + cc{k}_1)" for c, k in coef.items())
        w(f"  if constexpr (CM == CM_FMA) acc = R(2) * ({combo});  // x2 helicity flip")
        em.flops_per_level[0] += 3 * len(coef) + 1
    else:
        combo = " + ".join(f"cz{h}_{k}" for h in (0, 1) for k in range(ROW_ACCS))
        w(f"  if constexpr (CM == CM_FMA) acc = {combo};")
        em.flops_per_level[0] += 2 * ROW_ACCS - 1
    w("  return acc;")
    w("}")
    w("")
    # flops per event for the full helicity sum (one lane doing all helicities)
    total = 0
    for L in range(nlev):
        total += em.flops_per_level[L] * (2 ** L)
    w(f"// floating-point operations of one full helicity sum (all levels, all loop trips)")
    w(f"constexpr long FLOPS_HEL_SUM = {total};")
    w("}}  // namespace")
    emit_process.share_gaps = share_gaps
    return "\n".join(lines) + "\n", total


PROCESSES = {
    # name: (gluons on the top line, outgoing gluon indices, identical outgoing
    # gluons, hoist_weyl -- off for n = 4, whose live state already spills,
    # share_fp32 -- largest distance of a slash shared in FP32)
    "gg_tt": (2, (), 1, True, 8),
    "gg_ttg": (3, (2,), 1, True, 16),
    "gg_ttgg": (4, (2, 3), 2, False, 0),
}


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    out_dir = os.path.join(os.path.dirname(here), "csrc")
    for name, (n, outg, ident, hw, sh) in PROCESSES.items():
        src, fl = emit_process(name, n, outg, ident, hw, sh)
        with open(os.path.join(out_dir, f"gen_qcd_{name}.cuh"), "w") as f:
            f.write(src)
        print(name, "diagrams", diagram_count(n), "flops/hel-sum", fl)


if __name__ == "__main__":
    main()
