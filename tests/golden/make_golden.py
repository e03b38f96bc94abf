"""Writes the stored expected values under tests/golden/.

Every value is computed by the CPU oracle (package ``oracle``) on a seeded
input from ``graphgen``; nothing here touches the CUDA library.  Run from the
repository root:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def write(name, wl, source):
    dist, parent, pe = oracle.sssp(wl.row_ptr, wl.col, wl.weights, source)
    rec = {
        "workload": wl.name,
        "source": int(source),
        "input_sha256": digest(wl.row_ptr, wl.col, wl.weights),
        "dtype": str(wl.weights.dtype),
        "dist_bits": [int(x) for x in dist.view(np.uint32)],
        "parent": [int(x) for x in parent],
        "parent_edge": [int(x) for x in pe],
        "written_by": "tests/golden/make_golden.py (oracle.sssp: binary-heap Dijkstra + lowest-index parent rule)",
        "follows": "distances: the fixpoint of Algorithm 2 (Section 3.4), equal to the shortest-path distances of "
                   "Section 2.1 (fp32 weights as left-folded round-to-nearest sums, Section 4.2); parents: the "
                   "library's lowest-index tight-edge rule (the paper returns distances only)",
    }
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(rec, f)


if __name__ == "__main__":
    write("er1024_u32_src0.json", gg.tiny_er(), 0)
    wl = gg.grid_f32(32, 0.01, nsrc=1, seed=0)
    write("grid32_f32.json", wl, int(wl.sources[0]))
