"""Writes median27_net.h: the selection networks of the 3x3x3 median of the
denoise front end.

* sort9: sorts the 9 values of one plane's 3x3 neighbourhood.
* median3x9: the median (14th smallest) of 27 values given as three sorted
  lists of 9 (the neighbourhoods of planes z-1, z, z+1).

Each sorted plane list is used by three voxels along z, so a median costs
one sort9 and one median3x9.  Both networks start from Batcher's odd-even
merge sort (16 inputs with 7 held at +infinity for sort9; 64 inputs with
the three lists in the blocks starting at 0, 16 and 32 for median3x9) and
drop every comparator whose result follows from what is already known: a
+infinity input, the sorted order of the input lists, or the order earlier
comparators established.  median3x9 then keeps only the comparators its
output depends on, and a comparator one of whose outputs is not used keeps
only its min or its max.

Run: python gen_median27.py [output path]
"""
import os
import sys


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


def reduce(n, finite, sorted_groups):
    """Batcher's network on n wires without the comparators whose outcome is
    implied.  Returns (ops, var): ops are (lo, hi) variable pairs (after one,
    lo holds the min and hi the max) and var maps output wire -> variable."""
    le = [[i == j for j in range(n)] for i in range(n)]
    for grp in sorted_groups:
        for a in range(len(grp)):
            for b in range(a + 1, len(grp)):
                le[grp[a]][grp[b]] = True
    for w in range(n):
        if w not in finite:
            for k in range(n):
                le[k][w] = True

    def close():
        for k in range(n):
            lk = le[k]
            for i in range(n):
                if le[i][k]:
                    row = le[i]
                    for j in range(n):
                        if lk[j]:
                            row[j] = True

    close()
    var = list(range(n))
    ops = []
    for i, j in batcher(n):
        if le[i][j]:
            continue
        if le[j][i]:
            var[i], var[j] = var[j], var[i]
            le[i], le[j] = le[j], le[i]
            for row in le:
                row[i], row[j] = row[j], row[i]
            continue
        ops.append((var[i], var[j]))
        a, b = le[i][:], le[j][:]
        ka = [le[k][i] for k in range(n)]
        kb = [le[k][j] for k in range(n)]
        le[i] = [x or y for x, y in zip(a, b)]
        le[j] = [x and y for x, y in zip(a, b)]
        for k in range(n):
            le[k][i] = ka[k] and kb[k]
            le[k][j] = ka[k] or kb[k]
        le[i][j] = True
        le[j][i] = False
        le[i][i] = le[j][j] = True
        close()
    return ops, var


def sort9():
    ops, var = reduce(16, set(range(9)), [])
    return ops, [var[w] for w in range(9)]


def median3x9():
    finite = set(range(0, 9)) | set(range(16, 25)) | set(range(32, 41))
    groups = [list(range(0, 9)), list(range(16, 25)), list(range(32, 41))]
    ops, var = reduce(64, finite, groups)
    out = var[13]
    need, kept = {out}, []
    for a, b in reversed(ops):
        na, nb = a in need, b in need
        if na or nb:
            kept.append((a, b, na, nb))
            need.update((a, b))
    kept.reverse()
    return kept, out


def _cmp(lines, v, a, b, na=True, nb=True, mn="min", mx="max"):
    if na and nb:
        lines.append("    { const uint32_t t = %s(%s[%d], %s[%d]); %s[%d] = %s(%s[%d], %s[%d]); %s[%d] = t; }"
                     % (mn, v, a, v, b, v, b, mx, v, a, v, b, v, a))
    elif na:
        lines.append("    %s[%d] = %s(%s[%d], %s[%d]);" % (v, a, mn, v, a, v, b))
    else:
        lines.append("    %s[%d] = %s(%s[%d], %s[%d]);" % (v, b, mx, v, a, v, b))


def emit(path):
    s_ops, s_out = sort9()
    m_ops, m_out = median3x9()
    lines = [
        "// Generated by gen_median27.py: sort9 (%d comparators) and the median of" % len(s_ops),
        "// three sorted lists of 9 (%d comparators, pruned Batcher networks), on" % len(m_ops),
        "// one voxel per 32-bit word and on two voxels per word (16-bit halves).",
        "#pragma once",
        "",
        "// Sorts v[0..8] in place (s[k] receives the k-th smallest).",
        "__device__ __forceinline__ void sort9(const uint32_t *v, uint32_t *s) {",
        "    uint32_t w[16];",
    ]
    lines += ["    w[%d] = v[%d];" % (i, i) for i in range(9)]
    for a, b in s_ops:
        _cmp(lines, "w", a, b)
    lines += ["    s[%d] = w[%d];" % (k, s_out[k]) for k in range(9)]
    lines += ["}", "",
              "// The 14th smallest of a[0..8], b[0..8], c[0..8], each sorted ascending.",
              "__device__ __forceinline__ uint32_t median3x9(const uint32_t *a, const uint32_t *b, const uint32_t *c) {",
              "    uint32_t w[64];"]
    lines += ["    w[%d] = a[%d];" % (i, i) for i in range(9)]
    lines += ["    w[%d] = b[%d];" % (16 + i, i) for i in range(9)]
    lines += ["    w[%d] = c[%d];" % (32 + i, i) for i in range(9)]
    for a, b, na, nb in m_ops:
        _cmp(lines, "w", a, b, na, nb)
    lines += ["    return w[%d];" % m_out, "}"]
    # the same networks on two voxels at once: each 32-bit word holds two
    # 16-bit values and every comparator is one packed min and one packed max
    lines += ["",
              "// Packed unsigned 16-bit min and max of both halves (sm_90 and later).",
              "__device__ __forceinline__ uint32_t vmin16x2(uint32_t a, uint32_t b) {",
              "    uint32_t d;",
              '    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));',
              "    return d;",
              "}",
              "__device__ __forceinline__ uint32_t vmax16x2(uint32_t a, uint32_t b) {",
              "    uint32_t d;",
              '    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));',
              "    return d;",
              "}",
              "",
              "// sort9 on two voxels: every word of v holds one value of each.",
              "__device__ __forceinline__ void sort9x2(const uint32_t *v, uint32_t *s) {",
              "    uint32_t w[16];"]
    lines += ["    w[%d] = v[%d];" % (i, i) for i in range(9)]
    for a, b in s_ops:
        _cmp(lines, "w", a, b, mn="vmin16x2", mx="vmax16x2")
    lines += ["    s[%d] = w[%d];" % (k, s_out[k]) for k in range(9)]
    lines += ["}", "",
              "// median3x9 on two voxels (packed as in sort9x2).",
              "__device__ __forceinline__ uint32_t median3x9x2(const uint32_t *a, const uint32_t *b, const uint32_t *c) {",
              "    uint32_t w[64];"]
    lines += ["    w[%d] = a[%d];" % (i, i) for i in range(9)]
    lines += ["    w[%d] = b[%d];" % (16 + i, i) for i in range(9)]
    lines += ["    w[%d] = c[%d];" % (32 + i, i) for i in range(9)]
    for a, b, na, nb in m_ops:
        _cmp(lines, "w", a, b, na, nb, mn="vmin16x2", mx="vmax16x2")
    lines += ["    return w[%d];" % m_out, "}"]
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return len(s_ops), len(m_ops)


if __name__ == "__main__":
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                              "median27_net.h")
    print(emit(out))
