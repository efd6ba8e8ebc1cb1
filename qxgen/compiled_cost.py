"""Plan objective from the library's own compiled launch list (input generation only).

executed_time (qxgen.plan) estimates a plan from its pairwise steps alone;
the library's plan compiler also decides, per step, the kernel family, the
operand layouts and therefore the permutes, and which operands a launch
shares between its items.  CompiledTime compiles a plan on a host-only
handle (no GPU) and prices its launch list with
paper_2110_09894_gb300.cost.launch_list_time.
"""
from __future__ import annotations

from paper_2110_09894_gb300.cost import launch_list_time  # noqa: E402


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
