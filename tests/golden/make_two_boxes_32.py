"""Writes two_boxes_32.npz: the FP64 CPU oracle's pressure for the two-box
scene (two 0.3 x 0.5 x 0.3 boxes rotated 17 degrees about z, a 0.3-cell gap)
on a 32^3 grid with its seeded 32-mode Fourier velocity, solved directly
(sparse LU of the level-0 operator, Dirichlet p = 0 on y = 1).  Calls only the
oracle and the seeded scene generators.  The oracle build takes a few minutes,
so the GPU parity test reads this file instead of rebuilding it.

    python tests/golden/make_two_boxes_32.py
"""
import hashlib
import os
import sys

import numpy as np
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import scenes  # noqa: E402
from oracle.pipeline import build_system, rhs_full  # noqa: E402


def main():
    sc = scenes.config(1, 32)
    S = build_system(sc)
    V = S.meshes[0].V
    u = sc.velocity(V)
    r = rhs_full(S, u)
    p = np.zeros(len(V))
    p[S.free[0]] = spla.spsolve(S.H.A[0].tocsc(), r[S.free[0]])
    np.savez_compressed(os.path.join(HERE, "two_boxes_32.npz"), p=p,
                        v_sha256=np.frombuffer(hashlib.sha256(np.ascontiguousarray(V).tobytes()).digest(),
                                               dtype=np.uint8),
                        n_free=np.int64(len(S.free[0])))
    print("two_boxes_32.npz:", len(V), "vertices,", len(S.free[0]), "free DOFs")


if __name__ == "__main__":
    main()
