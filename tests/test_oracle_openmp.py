"""The OpenMP timing copy of the oracle (the CPU baseline on all host cores)
computes exactly what the plain single-threaded build computes: the loops it
spreads over threads are independent per node, so the states agree bit for
bit.  Also: the reference arm's timing helper runs on it."""
import numpy as np
import pytest

from paper_1710_07486_gb300 import inputs
from tests.cases import A, B, RGAS, asymmetric


@pytest.mark.parametrize("lattice,shape", [(0, (40, 36, 1)), (1, (14, 12, 10))])
def test_openmp_build_is_bitwise_the_plain_build(orc, lattice, shape):
    try:
        orc.build(openmp=True)
    except Exception as ex:  # no OpenMP in this compiler: nothing to compare
        pytest.skip(f"no OpenMP build: {ex}")
    T = orc.temperature_for_ratio(A, B, RGAS, 10.0)
    p = asymmetric(T, gamma_mode=1)
    D = 2 if lattice == 0 else 3
    dims = shape[:D]
    states = []
    for omp in (False, True):
        o = orc.Oracle(lattice, *shape, p, openmp=omp)
        c = [v / 2.0 for v in dims]
        rho, phi, u = inputs.drops(dims, o.rho_g, o.rho_l, p["chi"],
                                   [dict(center=[v - 3 for v in c], R=min(dims) / 4, kind=1, u=[0.02] * D),
                                    dict(center=[v + 3 for v in c], R=min(dims) / 5, kind=-1)], width=4.0)
        f, g = o.init(rho, phi, u)
        assert o.step(f, g, 4) == 0
        states.append((f, g, o.fields(f, g)["p"]))
    for a, b in zip(states[0], states[1]):
        assert np.array_equal(a, b)


def test_reference_timing_helper_runs(orc):
    import bench
    v, done, dt = bench.oracle_run(8, 1, 1710, openmp=False)
    assert done == 1 and v > 0 and dt > 0
