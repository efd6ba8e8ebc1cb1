"""Time estimate of a contraction call from the library's compiled launch list.

The plan compiler decides, for every pairwise step, the kernel family, the
operand layouts (and so the permutes) and which operands a launch shares
between its items; qx_describe_plan lists those launches.  This prices each
listed launch on one GB300: its bytes (operands read once per item, an
operand of a lower dependence level once per launch, the result written
once) at the HBM rate its kernel family reaches, or its complex flops
(8 M K N) at the family's arithmetic rate, whichever takes longer, plus a
launch cost, and sums the launches.  The rates were measured per family on
the 36-qubit sliced workload, where the sum matched the measured step time
(325 vs 326 ms in 3xTF32, and again after the kernels changed).  The server uses it for admission, planners to
rank plans.
"""
from __future__ import annotations

# kernel family -> (complex flop/s, or None for data movement; bytes/s).  "tc_direct_kb": the direct
# tensor-core kernel with B' resident per CTA (B shared by every item, one tile wide)
GB300_LAUNCH_RATES = {"permute": (None, 6.0e12), "gather": (26e12, 4.7e12), "tc_direct": (150e12, 3.5e12),
                      "tc_direct_kb": (150e12, 4.8e12), "tc_prep": (260e12, 5.0e12), "gemm": (35e12, 4.0e12),
                      "dot_perm": (35e12, 5.0e12)}
_LEVEL = {"shared": 0, "slice": 1, "pair": 2}


def _regions(field):
    out = []
    for part in field.split(",") if field else ():
        reg, rest = part.split(":")
        out.append((reg, int(rest.split("+")[1])))
    return out


def launch_list_time(desc, n_slices, n_bits, rates=GB300_LAUNCH_RATES, launch=4e-6):
    """Seconds of one call over n_slices slices and n_bits bitstrings from a qx_describe_plan listing
    (launches priced one after another)."""
    items = (1, n_slices, n_slices * n_bits)
    total = 0.0
    for line in desc.splitlines():
        f = line.split()
        kind, level = f[2], _LEVEL[f[3]]
        kv = dict(x.split("=", 1) for x in f[4:] if "=" in x)
        it = items[level]
        nbytes = sum(8.0 * e * (it if _LEVEL[r] == level else items[_LEVEL[r]]) for r, e in _regions(kv.get("reads", "")))
        nbytes += sum(8.0 * e * it for r, e in _regions(kv.get("writes", "")))
        if kind == "tc_direct" and "m" in kv:
            # the launch picks the resident-B' variant when B is shared by every item, one 128- or 64-wide
            # tile (N = 64 or 32) and at most 4 or 8 K stages of 32 reals, and A is not kept per slice
            regs = _regions(kv.get("reads", ""))
            n, k = int(kv["n"]), int(kv["k"])
            if len(regs) == 2 and regs[1][0] == "shared" and regs[0][0] == f[3] and (
                    (n == 6 and (2 << k) // 32 <= 4) or (n == 5 and (2 << k) // 32 <= 8)):
                kind = "tc_direct_kb"
        fr, br = rates.get(kind, (35e12, 4.0e12))
        t = nbytes / br
        if fr and "m" in kv:
            t = max(t, 8.0 * 2.0 ** (int(kv["m"]) + int(kv["k"]) + int(kv["n"])) * it / fr)
        total += t + launch
    return total
