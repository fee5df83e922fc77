"""Context checks of the oracle against numbers printed in the paper."""
import json
import os

import oracle as O
import vie_synth as V

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_gmres_iterations.json")


def test_gmres_iterations_homogeneous_table():
    # Table TAB:Con Coeff prints 10 GMRES iterations at every N for mu_s = 2,
    # mu = 2.2, tolerance 1e-12.  With a stand-in source the count must be
    # close to 10 and independent of the mesh.
    g = json.load(open(GOLDEN))
    its = []
    for n in (16, 32):
        m = V.homogeneous_medium(2, n, g["mu"], g["mu_s"])
        phi = O.apply(2, m.sigma_t, m.sigma_s, m.f, op=O.OP_A_RAW, mode=O.TAU_CLOSED)
        U, it, rr, ok = O.gmres(2, m.sigma_t, m.sigma_s, phi, rtol=g["tol"], mode=O.TAU_CLOSED)
        assert ok
        its.append(it)
    assert abs(its[0] - its[1]) <= 1
    assert all(abs(i - g["iterations"][0]) <= 2 for i in its)
