"""Write the converged-energy golden values used by the GPU parity tests.

Calls only the CPU oracle.  Each workload is run from the same seeded
orbitals until the energy stops changing at the 1e-13 level; both
Barzilai-Borwein variants (tau1 and alternating) must agree, which pins the
minimum independently of the trajectory.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pou_oracle as O  # noqa: E402
from paper_1510_07230_gb300 import inputs  # noqa: E402


def converged_energy(name, bb, max_iter):
    w, R, Z, U0 = inputs.workload_inputs(name)
    cfg = O.cubic(w.n, w.L, order=w.order, N=w.N, bb_variant=bb)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    st = O.run(U0, vext, cfg, max_iter)
    E = [h.energy for h in st.history]
    HW = O.apply_h(st.W, st.V, cfg)
    return min(E), O.gradient_residual(st.W, HW, cfg), len(E)


def main():
    out = {}
    name = "l10_g32_n4"
    e3, g3, n3 = converged_energy(name, 3, 3000)
    e1, g1, n1 = converged_energy(name, 1, 6000)
    assert abs(e3 - e1) < 1e-10, (e3, e1)
    out[name] = {"E_converged": e3, "grad_norm_bb3": g3, "iterations_bb3": n3,
                 "E_converged_bb1": e1, "grad_norm_bb1": g1, "iterations_bb1": n1,
                 "source": "oracle/pou_oracle.py run to convergence (tests/golden/make_golden.py)"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "converged_energies.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
