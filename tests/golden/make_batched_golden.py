"""Write the state-vector amplitudes of the 256 circuits of the batched uneven workload.

Calls only the oracle (complex128 state-vector evolution in C, Sec. II) on the
seeded circuits and bitstrings of qxgen.workloads.batched_circuit_greedy (the
circuits and bitstrings do not depend on the plan).  Circuits of up to 28
qubits need 4 GiB each and about a minute or two of host time; the whole
set takes about an hour on 8 cores.  Output: batched_statevector.json next to
this file, one record per circuit with a digest of its gates and bitstrings.

    python tests/golden/make_batched_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from qxgen import workloads  # noqa: E402


def case_digest(w):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(w.gates).tobytes())
    h.update(np.asarray(w.bitstrings, np.uint8).tobytes())
    h.update(np.asarray(w.open_mask, np.uint8).tobytes())
    return h.hexdigest()


def main(path=os.path.join(HERE, "batched_statevector.json")):
    done = {}
    if os.path.exists(path):  # resume: keep records whose circuit is unchanged
        with open(path) as f:
            done = {r["j"]: r for r in json.load(f)["circuits"]}
    out = []
    for j in range(256):
        w = workloads.batched_circuit_greedy(j)
        dg = case_digest(w)
        if j in done and done[j]["digest"] == dg:
            out.append(done[j])
            continue
        a = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
        out.append({"j": j, "name": w.name, "digest": dg, "re": a.real.tolist(), "im": a.imag.tolist()})
        with open(path + ".tmp", "w") as f:
            json.dump({"source": "oracle.sv_amplitudes (complex128 state vector)", "circuits": out}, f)
        os.replace(path + ".tmp", path)
        print(j, w.name, flush=True)
    with open(path, "w") as f:
        json.dump({"source": "oracle.sv_amplitudes (complex128 state vector)", "circuits": out}, f)


if __name__ == "__main__":
    main()
