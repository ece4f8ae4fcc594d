"""FoF catalogue (Sec. IV-B) against the oracle's catalogue: group order
(bit-exact), group labels, counts, offsets and masses (exact), centre of mass,
velocity and inertia radius (float64 sums rounded to float32)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from tests import parity
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _compare(x, L, vel, b, min_count, pmass):
    import paper_2604_05885_gb300 as jzt
    tree = jzt.build(to_dev(x), periodic_L=L)
    labels, order, groups = tree.fof_catalogue(b, vel=None if vel is None else to_dev(vel), min_count=min_count,
                                               particle_mass=pmass)
    lab = labels.cpu().numpy()
    s, lo = oracle.fof_bracket(x, b, L, cells=False)
    parity.check_fof(lab, s, lo)
    ro, rg = oracle.fof_catalogue(x, lab, L, vel=vel, min_count=min_count, particle_mass=pmass)
    assert np.array_equal(order.cpu().numpy(), ro)
    assert len(groups) == len(rg)
    for g, r in zip(groups, rg):
        assert (int(g["label"]), int(g["count"]), int(g["offset"])) == (r["label"], r["count"], r["offset"])
        assert np.float32(g["mass"]) == np.float32(r["mass"])
        assert np.allclose(g["x_cm"], r["x_cm"], rtol=0, atol=2e-7), (g, r)
        assert np.allclose(g["v_cm"], r["v_cm"], rtol=1e-6, atol=1e-6), (g, r)
        assert abs(float(g["r_inertia"]) - r["r_inertia"]) <= 2e-7 * max(1.0, r["r_inertia"]) + 1e-7 * r["r_inertia"]
    return groups


@pytest.mark.parametrize("L", [1.0, 0.0])
@pytest.mark.parametrize("min_count", [20, 3])
def test_catalogue_clustered(L, min_count):
    n = 20000
    x = workloads.clustered(n, 61, n_blobs=40)
    vel = np.random.default_rng(62).standard_normal((n, 3)).astype(np.float32)
    groups = _compare(x, L, vel, 0.25 * workloads.mean_spacing(n), min_count, 1.5)
    assert len(groups) > 5


def test_catalogue_singletons_and_no_velocity():
    x = workloads.uniform(5000, 63)
    _compare(x, 1.0, None, 0.05 * workloads.mean_spacing(5000), 1, 1.0)


def test_catalogue_group_across_periodic_boundary():
    # a dense blob centred on a box corner: its members wrap around all three faces
    rng = np.random.default_rng(64)
    x = workloads.snap_unit(rng.normal(0.0, 0.004, (3000, 3)))
    _compare(x, 1.0, None, 0.004, 20, 1.0)


def test_catalogue_capacity_error():
    import paper_2604_05885_gb300 as jzt
    x = workloads.clustered(8000, 65, n_blobs=30)
    tree = jzt.build(to_dev(x), periodic_L=1.0)
    with pytest.raises(jzt.JztError) as e:
        tree.fof_catalogue(0.3 * workloads.mean_spacing(8000), min_count=2, cap_groups=1)
    assert e.value.code == jzt.JZT_ERR_CAPACITY
    torch.cuda.synchronize()
