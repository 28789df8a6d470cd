"""Writes median27_net.h: a branch-free selection network for the median of
27 values (the 14th smallest), used by the 3x3x3 median of the denoise
front end.

Construction: Batcher's odd-even merge sort network on 32 inputs, with the
inputs 27..31 held at +infinity.  A comparator whose upper input is known
to be +infinity never exchanges and is dropped; one whose lower input is
+infinity always exchanges and becomes a renaming.  Then only the
comparators on which output 13 depends are kept, and a comparator one of
whose outputs is not used afterwards keeps only its min or its max.

Run: python gen_median27.py [output path]
"""
import os
import sys

N, N_REAL, OUT = 32, 27, 13


def batcher(n):
    comps = []
    p = 1
    while p < n:
        k = p
        while k >= 1:
            j = k % p
            while j <= n - 1 - k:
                for i in range(0, min(k - 1, n - j - k - 1) + 1):
                    if (i + j) // (p * 2) == (i + j + k) // (p * 2):
                        comps.append((i + j, i + j + k))
                j += 2 * k
            k //= 2
        p *= 2
    return comps


def network():
    var = list(range(N))            # wire -> variable name index
    inf = [w >= N_REAL for w in range(N)]
    ops = []                        # (lo_var, hi_var) in program order
    for i, j in batcher(N):
        if inf[j]:
            continue
        if inf[i]:
            var[i], var[j] = var[j], var[i]
            inf[i], inf[j] = inf[j], inf[i]
            continue
        ops.append((var[i], var[j]))
    # after a comparator (a, b): variable a holds the min, b the max
    out_var = var[OUT]
    need = {out_var}
    kept = []
    for a, b in reversed(ops):
        na, nb = a in need, b in need
        if not (na or nb):
            continue
        kept.append((a, b, na, nb))
        need.add(a)
        need.add(b)
    kept.reverse()
    return kept, out_var


def emit(path):
    kept, out_var = network()
    lines = [
        "// Generated by gen_median27.py: median (14th smallest) of 27 values by",
        "// a pruned odd-even merge network (%d comparators)." % len(kept),
        "#pragma once",
        "",
        "__device__ __forceinline__ uint32_t median27_net(uint32_t *v) {",
    ]
    for a, b, na, nb in kept:
        if na and nb:
            lines.append("    { const uint32_t t = min(v[%d], v[%d]); v[%d] = max(v[%d], v[%d]); v[%d] = t; }"
                         % (a, b, b, a, b, a))
        elif na:
            lines.append("    v[%d] = min(v[%d], v[%d]);" % (a, a, b))
        else:
            lines.append("    v[%d] = max(v[%d], v[%d]);" % (b, a, b))
    lines.append("    return v[%d];" % out_var)
    lines.append("}")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return len(kept)


if __name__ == "__main__":
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                              "median27_net.h")
    print(emit(out))
