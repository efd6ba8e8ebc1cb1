"""Time estimate of a plan from the library's own compiled launch list (input generation only).

executed_time (qxgen.plan) estimates a plan from its pairwise steps alone;
the library's plan compiler also decides, per step, the kernel family, the
operand layouts and therefore the permutes, and which operands a launch
shares between its items.  This estimate compiles the plan on a host-only
handle (no GPU) and prices every launch that qx_describe_plan lists: its
bytes (operands read once per item, an operand of a lower level once per
launch, the result written once) at the HBM rate its kernel family reaches,
or its flops at the family's arithmetic rate, whichever takes longer, plus a
launch cost.  The rates are the ones measured on GB300 for each family on
the 36-qubit workload; this sum matched that workload's measured step time
(325 vs 326 ms) and its per-family split.
"""
from __future__ import annotations

# kernel family -> (complex flop/s in the 8 M K N convention, or None for data movement; bytes/s)
GB300_LAUNCH_RATES = {"permute": (None, 6.0e12), "gather": (20e12, 4.7e12), "tc_direct": (150e12, 4.0e12),
                      "tc_prep": (174e12, 5.0e12), "gemm": (35e12, 4.0e12), "dot_perm": (35e12, 5.0e12)}
_LEVEL = {"shared": 0, "slice": 1, "pair": 2}


def _regions(field):
    out = []
    for part in field.split(",") if field else ():
        reg, rest = part.split(":")
        out.append((reg, int(rest.split("+")[1])))
    return out


def launch_list_time(desc, n_slices, n_bits, rates=GB300_LAUNCH_RATES, launch=4e-6):
    """Seconds of one call from a qx_describe_plan listing (launches priced one after another)."""
    items = (1, n_slices, n_slices * n_bits)
    total = 0.0
    for line in desc.splitlines():
        f = line.split()
        kind, level = f[2], _LEVEL[f[3]]
        kv = dict(x.split("=", 1) for x in f[4:] if "=" in x)
        it = items[level]
        nbytes = sum(8.0 * e * (it if _LEVEL[r] == level else items[_LEVEL[r]]) for r, e in _regions(kv.get("reads", "")))
        nbytes += sum(8.0 * e * it for r, e in _regions(kv.get("writes", "")))
        fr, br = rates.get(kind, (35e12, 4.0e12))
        t = nbytes / br
        if fr and "m" in kv:
            t = max(t, 8.0 * 2.0 ** (int(kv["m"]) + int(kv["k"]) + int(kv["n"])) * it / fr)
        total += t + launch
    return total


class CompiledTime:
    """Callable objective for qxgen.plan.local_search_plan: the launch-list time of a plan compiled by
    libqx for one network (built once on a host-only handle) in one precision form."""

    def __init__(self, n_qubits, gate_records, open_mask, precision=1):
        from paper_2110_09894_gb300 import qx
        self.qx = qx
        self.h = qx.qx_create(-1, precision=precision)
        qx.qx_build_network(self.h, n_qubits, gate_records, open_mask)

    def __call__(self, legs, order, sliced, n_outputs, n_bits):
        self.qx.qx_set_plan(self.h, order, sliced)
        return launch_list_time(self.qx.qx_describe_plan(self.h), 1 << len(sliced), n_bits)

    def close(self):
        if self.h is not None:
            self.qx.qx_destroy(self.h)
            self.h = None
