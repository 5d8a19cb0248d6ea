"""Build-time generator of the helicity-summed amplitude of e- e+ -> n photons.

Pure QED with massless electrons: the n! tree diagrams attach the photons to
the electron line in every order.  Summed over orders, the off-shell electron
spinor with a set T of photons attached obeys the Berends-Giele recursion

    S(T) = Sprop(p0 - k_T) sum_{i in T} eps*_i-slash S(T \\ {i}),   S({}) = u(p0),

and the amplitude is  A = vbar(p1) sum_i eps*_i-slash S(all \\ {i})  (the same
sum of diagrams, every sub-chain shared): 2^n - 2 spinors instead of n! n
chain links.  Massless spinors keep one chirality, so every S(T) is a
two-component right-handed Weyl spinor, and eps-slash / the propagator swap
the two 2x2 blocks of the chiral-basis Dirac matrices.

The helicity sum is written as nested loops over the photon helicities, every
S(T) computed at the outermost loop level on which it depends (the level of
its highest photon); the electron helicity is fixed and the sum doubled
(flipping every helicity conjugates the amplitude).  Couplings are stripped
(e = 1): |M|^2 = e^(2n) * (returned sum) / (4 n!).

Run ``python -m paper_2312_07440_gb300.gen.qed_gen`` to regenerate
``csrc/gen_qed_ee_5a.cuh`` (the generated header is committed).
"""
from __future__ import annotations

import math
import os

# floating-point operations of the emitted building blocks (FMA = 2)
FLOPS = {
    "sl": 28,      # eps-slash on a 2-spinor: 4 complex products, 2 complex sums
    "acc": 4,      # adding a 2-spinor
    "pr": 20,      # propagator (real 2x2 blocks, pre-scaled by 1/q^2) on a 2-spinor
    "close": 14,   # vbar . psi
    "abs2": 4,     # |A|^2 accumulated
}


def popcount(m):
    return bin(m).count("1")


def emit_process(name, n):
    full = (1 << n) - 1
    lines = []
    w = lines.append
    flops_level = [0] * n
    w(f"// ---- generated by gen/qed_gen.py: {name} (e- e+ -> {n} photons), do not edit ----")
    w(f"// {math.factorial(n)} Feynman diagrams, {2 ** (n + 2)} helicities; "
      f"{full - 1} off-shell electron spinors per helicity configuration.")
    w("#pragma once")
    w('#include "qed.cuh"')
    w("")
    w(f"namespace rw {{ namespace {name} {{")
    w(f"constexpr int NA = {n};")
    w(f"constexpr int NEXT = {n + 2};")
    w(f"constexpr int NHEL = {2 ** (n + 2)};")
    w(f"constexpr int NDIAG = {math.factorial(n)};")
    w(f"constexpr int MAX_LB = {n};  // helicity levels that can be spread over lanes")
    w(f"constexpr int IDENT = {n};  // identical photons (1/IDENT!)")
    w("")
    w("// Sum over this lane's photon helicities of |A|^2 (e = 1), electron helicity")
    w("// fixed and doubled.  Levels 0..LB-1 (photons 0..LB-1) take their helicity from")
    w("// the lane index, the others loop.")
    w("template <class R, int LB>")
    w(f"__device__ __forceinline__ R hel_sum(const QedExt<R, NA>& X, const QedKin<R, NA>& Kn, int lane) {{")
    w("  R acc = R(0);")
    w("  const w2<R> S0 = X.u;")
    ind = "  "

    def sname(m):
        return f"S{m}"

    for L in range(n):
        bit = f"((lane >> (LB - 1 - {L})) & 1)"
        w(f"{ind}#pragma unroll 1")
        w(f"{ind}for (int i{L} = 0; i{L} < (LB > {L} ? 1 : 2); ++i{L}) {{")
        ind += "  "
        w(f"{ind}const int h{L} = LB > {L} ? {bit} : i{L};")
        w(f"{ind}const ws<R>& E{L} = X.eps[{L}][h{L}];")
        # spinors whose highest photon is L, by increasing size
        masks = sorted((m for m in range(1, full) if m.bit_length() - 1 == L), key=lambda m: (popcount(m), m))
        for m in masks:
            terms = [i for i in range(n) if (m >> i) & 1]
            w(f"{ind}w2<R> t{m} = sl_RL(E{terms[0]}, {sname(m & ~(1 << terms[0]))});")
            flops_level[L] += FLOPS["sl"]
            for i in terms[1:]:
                w(f"{ind}sl_RL_acc(t{m}, E{i}, {sname(m & ~(1 << i))});")  # fused accumulation
                flops_level[L] += FLOPS["sl"] + FLOPS["acc"]
            w(f"{ind}const w2<R> {sname(m)} = pr_LR(Kn.q[{m}], t{m});")
            flops_level[L] += FLOPS["pr"]
        if L == n - 1:
            # close the line: A = vbar . sum_i eps_i-slash S(all \ i)
            w(f"{ind}w2<R> T = sl_RL(E0, {sname(full & ~1)});")
            flops_level[L] += FLOPS["sl"]
            for i in range(1, n):
                w(f"{ind}sl_RL_acc(T, E{i}, {sname(full & ~(1 << i))});")
                flops_level[L] += FLOPS["sl"] + FLOPS["acc"]
            w(f"{ind}const cx<R> A = close_L(X.vb, T);")
            w(f"{ind}acc += A.r * A.r + A.i * A.i;")
            flops_level[L] += FLOPS["close"] + FLOPS["abs2"]
    for L in range(n - 1, -1, -1):
        ind = ind[:-2]
        w(f"{ind}}}")
    w("  return R(2) * acc;  // x2: the other electron helicity (all helicities flipped)")
    w("}")
    w("")
    total = sum(f * 2 ** (L + 1) for L, f in enumerate(flops_level))
    w("// floating-point operations of one full helicity sum (all levels, all loop trips)")
    w(f"constexpr long FLOPS_HEL_SUM = {total};")
    w("}}  // namespace")
    return "\n".join(lines) + "\n", total


PROCESSES = {"ee_5a": 5}


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    out_dir = os.path.join(os.path.dirname(here), "csrc")
    for name, n in PROCESSES.items():
        src, fl = emit_process(name, n)
        with open(os.path.join(out_dir, f"gen_qed_{name}.cuh"), "w") as f:
            f.write(src)
        print(name, "diagrams", math.factorial(n), "flops/hel-sum", fl)


if __name__ == "__main__":
    main()
