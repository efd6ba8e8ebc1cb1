"""Write the oracle's partial sum over slices 0..31 of the 6x6 depth-14 workload.

Calls only the oracle (complex128 plan einsum, compensated slice sum) on the
seeded workload from qxgen.workloads.large(); about 30 s of CPU per slice
group of 8 on a few cores.  Output: large_slices0_31.json next to this file,
with a digest of the plan so a changed planner is detected instead of
silently compared against stale values.

    python tests/golden/make_large_golden.py
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


def main(n_slices=32):
    w = workloads.large()
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
    with open(os.path.join(HERE, f"large_slices0_{n_slices - 1}.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
