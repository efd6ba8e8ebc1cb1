"""Write the oracle's partial sum over slices 0..31 of the 6x6 depth-14 workload.

Calls only the oracle (complex128 plan einsum, compensated slice sum) on the
seeded workload: `greedy` follows qxgen.workloads.large() (its seeded greedy
order; several minutes of CPU) into large_slices0_31.json, `ls` follows
qxgen.workloads.large_local_search() (the stored local-search order of the
same sliced bonds; about a minute) into large_ls_slices0_31.json, `sa`
follows qxgen.workloads.large_annealed() (the stored annealed plan, which
slices other bonds) into large_sa_slices0_31.json.  Each file
carries a digest of its plan so a changed planner is detected instead of
silently compared against stale values.  The two orders contract the same 32
sub-networks (Eq. 2), so the two files agree to complex128 rounding; the
annealed plan's slices 0..31 are other sub-networks, so its file holds
another partial sum.

    python tests/golden/make_large_golden.py [greedy] [ls] [sa]
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import einsum  # noqa: E402
from qxgen import workloads  # noqa: E402


def plan_digest(w):
    h = hashlib.sha256()
    h.update(np.asarray(w.order, np.int64).tobytes())
    h.update(np.asarray(w.sliced, np.int64).tobytes())
    h.update(np.ascontiguousarray(w.gates).tobytes())
    h.update(np.asarray(w.bitstrings, np.uint8).tobytes())
    return h.hexdigest()


def main(which="greedy", n_slices=32):
    w = {"greedy": workloads.large, "ls": workloads.large_local_search, "sa": workloads.large_annealed}[which]()
    amps = einsum.amplitudes(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, w.bitstrings,
                             slices=range(n_slices))
    out = {
        "workload": w.name,
        "slices": [0, n_slices],
        "plan_sha256": plan_digest(w),
        "bitstring": "".join(str(int(b)) for b in w.bitstrings[0]),
        "re": amps[0].real.tolist(),
        "im": amps[0].imag.tolist(),
        "source": "oracle.einsum.amplitudes (complex128, Neumaier slice sum)",
    }
    name = f"large_slices0_{n_slices - 1}.json" if which == "greedy" else f"large_{which}_slices0_{n_slices - 1}.json"
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    for which in sys.argv[1:] or ["greedy", "ls"]:
        main(which)
