"""Write the stored expected values of the GPU tests.  Calls only the FP64 CPU oracle
(oracle/) on the seeded synthetic inputs (synth/); nothing here comes from the CUDA path.

  config2_converged_T.txt   radiative-equilibrium profile of the full-size single atmosphere
                            (100 layers x 3000 bins x 20 g, Rayleigh-like scattering), converged
                            by the oracle to |dF|/(sigma T^4) < 1e-9 from the isothermal start.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402


def config2_profile(tol=1e-9):
    wl = synth.config2()
    atm = oracle.Atm.from_workload(wl)
    st = oracle.State(atm, wl.atms[0].T_init)
    t0 = time.time()
    rc, it, m = oracle.solve_re(atm, st, oracle.params(tol=tol, max_iter=200000))
    assert rc == oracle.CONVERGED, (rc, it, m)
    hdr = (f"oracle radiative-equilibrium profile, config {wl.name}, tol {tol:g}, {it} flux evaluations, "
           f"final metric {m:.3e}, {time.time() - t0:.0f} s\nlayer 0 = bottom; K")
    np.savetxt(os.path.join(HERE, "config2_converged_T.txt"), st.T, fmt="%.10f", header=hdr)


if __name__ == "__main__":
    config2_profile()
