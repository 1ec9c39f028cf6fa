"""Source iteration of small 1D problems with two warps per cell (one block
a cell: the two faces evaluated by different warps and exchanged, the
Planck values and the opacities evaluated side by side) against one warp
per cell: the same operations on the same operands, so the same bits in T,
rho and the iterate count, step after step."""
import numpy as np
import pytest

from paper_2312_16981_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2312_16981_gb300 import binding
    binding.load()
    return binding


def run(B, p, steps):
    sim = B.Simulation(p)
    out = []
    for _ in range(steps):
        sim.step(1)
        t = sim.tallies()
        assert t["status_bits"] == 0
        g = sim.get_state()
        out.append((g["T"], g["rho"], t["si_iters"]))
    return out


@pytest.mark.parametrize("case", ["slab_fp64", "slab_mixed", "larsen", "olson", "many_groups"])
def test_pair_equals_one_warp_per_cell(B, case):
    if case.startswith("slab"):
        p = I.small_multigroup(nx=24, G=6, omega_ref=1e-6)
        if case == "slab_mixed":
            p = p.replace(precision=I.MIXED)
    elif case == "larsen":
        p = I.larsen_slab(G=12, omega_frac=2e-5)
    elif case == "olson":
        p = I.olson_slab(G=10, omega_frac=1e-3)
    else:
        # two groups per lane (G > 32) and a reflecting far side
        p = I.multigroup_slab(nx=40, G=40, omega_ref=1e-6)
        p.particle_capacity = 1 << 20
    a = run(B, p.replace(si_pair=0), 4)
    b = run(B, p.replace(si_pair=-1), 4)
    for (Ta, ra, ia), (Tb, rb, ib) in zip(a, b):
        np.testing.assert_array_equal(Ta, Tb)
        np.testing.assert_array_equal(ra, rb)
        assert ia == ib
