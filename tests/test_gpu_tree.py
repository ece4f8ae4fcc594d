"""Tree construction parity (Sec. II) against the oracle, bit-exact: Morton keys,
stable sort order, gathered points, plane splits, node counts and boxes."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _gauss_outliers(seed=7):
    rng = np.random.default_rng(seed)
    return workloads.clip_unit(np.concatenate([rng.normal(0.5, 0.01, (6000, 3)), rng.random((60, 3))]))


def _cases():
    x_dup = workloads.uniform(3000, 4)
    x_dup[100:400] = x_dup[100]          # a run of 300 identical points
    x_dup[1000:1040] = x_dup[7]
    x_line = np.zeros((700, 3), np.float32)
    x_line[:, 0] = workloads.uniform(700, 5)[:, 0]
    return [
        ("uniform-open", workloads.uniform(5000, 1), 0.0, None),
        ("uniform-periodic", workloads.uniform(4099, 2), 1.0, None),
        ("clustered-periodic-3planes", workloads.clustered(20000, 3, n_blobs=30), 1.0,
         dict(n_target=10)),
        ("duplicates", x_dup, 0.0, dict(nmax0=8, plane_factor=4, n_target=4)),
        ("line", x_line, 0.0, dict(nmax0=4, plane_factor=2, n_target=8)),
        ("lattice", workloads.lattice(9), 1.0, dict(nmax0=16)),
        ("tiny-1", workloads.uniform(1, 6), 0.0, None),
        ("tiny-2", workloads.uniform(2, 6), 1.0, None),
        ("tiny-33", workloads.uniform(33, 6), 0.0, None),
        ("ragged-tiles", workloads.uniform(4096 * 3 + 17, 8), 0.0, dict(nmax0=5, n_target=30)),
        # regularisation (Sec. II-D): a dense Gaussian with far outliers, and the duplicates case
        ("reg-gauss-outliers", _gauss_outliers(), 0.0, dict(n_target=20, reg_fmax=50.0)),
        ("reg-gauss-periodic", _gauss_outliers(8), 1.0, dict(nmax0=16, n_target=8, reg_fmax=4.0)),
        ("reg-duplicates", x_dup, 0.0, dict(nmax0=8, plane_factor=4, n_target=4, reg_fmax=1.0)),
    ]



@pytest.mark.parametrize("name,x,L,params", _cases(), ids=[c[0] for c in _cases()])
def test_tree_matches_oracle(name, x, L, params):
    import paper_2604_05885_gb300 as jzt
    p = dict(params or {})
    nmax0 = p.get("nmax0", 32)
    c = p.get("plane_factor", 8)
    nt = p.get("n_target", 1000)
    tree = jzt.build(to_dev(x), periodic_L=L, params=p or None)
    st = tree.status()
    assert st["code"] == 0, st
    keys, pts, n_planes = tree.arrays()
    assert n_planes == oracle.num_planes(len(x), nmax0, c, nt)
    ref_keys = oracle.morton_keys(x, L)
    sk, perm = oracle.zsort(ref_keys)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), sk)
    p_np = pts.cpu().numpy()
    assert np.array_equal(p_np[:, 3].view(np.int32), perm.astype(np.int32))
    assert np.array_equal(p_np[:, :3], x[perm])
    spl_ref, gaps_ref = oracle.plane_splits(sk, nmax0=nmax0, c=c, n_target=nt, f_max=p.get("reg_fmax", 0.0))
    if p.get("reg_fmax"):
        plain = oracle.plane_splits(sk, nmax0=nmax0, c=c, n_target=nt)[1]
        assert any(len(a) != len(b) for a, b in zip(gaps_ref, plain)), "regularisation added no split"
    nodes_ref = oracle.plane_nodes(x[perm], gaps_ref)
    for pl in range(n_planes):
        spl, cnt, box = tree.plane(pl)
        assert np.array_equal(spl, spl_ref[pl].astype(np.int32)), f"plane {pl} splits"
        rc, rlo, rhi = nodes_ref[pl]
        assert np.array_equal(cnt, rc.astype(np.int32)), f"plane {pl} counts"
        assert np.array_equal(box[:, :3], rlo) and np.array_equal(box[:, 3:], rhi), f"plane {pl} boxes"


def test_invalid_coordinates_set_input_status():
    import paper_2604_05885_gb300 as jzt
    x = workloads.uniform(1000, 9)
    x[17, 1] = np.nan
    tree = jzt.build(to_dev(x), periodic_L=0.0)
    assert tree.status()["code"] == jzt.JZT_ERR_INPUT
    x = workloads.uniform(1000, 9)
    x[3, 0] = 1.0  # outside [0, L) for L = 1
    tree = jzt.build(to_dev(x), periodic_L=1.0)
    assert tree.status()["code"] == jzt.JZT_ERR_INPUT


def test_regularisation_leaves_results_unchanged():
    """Sec. II-D: the regularisation changes the tree only, never the kNN rows or FoF labels."""
    import paper_2604_05885_gb300 as jzt
    x = _gauss_outliers(11)
    for L in (0.0, 1.0):
        a = jzt.build(to_dev(x), periodic_L=L)
        r = jzt.build(to_dev(x), periodic_L=L, params=dict(reg_fmax=50.0))
        ia, da = a.knn(16)
        ir, dr = r.knn(16)
        assert np.array_equal(ia.cpu().numpy(), ir.cpu().numpy())
        assert np.array_equal(da.cpu().numpy(), dr.cpu().numpy())
        b = 0.3 * workloads.mean_spacing(len(x))
        assert np.array_equal(a.fof(b).cpu().numpy(), r.fof(b).cpu().numpy())


def _bucket_cases():
    x_dup = workloads.uniform(1 << 17, 21)
    x_dup[5000:5300] = x_dup[5000]       # 300 equal keys: the index passes restore input order
    x_dup[90000:90007] = x_dup[12]       # equal keys written far apart in the input
    x_heavy = workloads.uniform(1 << 17, 23)
    x_heavy[:3000] = x_heavy[77]         # one fine bin above 2048 keys: the LSD passes run
    rng = np.random.default_rng(24)      # a dense blob: one bin of ~1500 distinct keys (block sort)
    x_blob = workloads.uniform(1 << 17, 24)
    x_blob[:1500] = workloads.clip_unit(rng.normal(0.3, 5e-5, (1500, 3)))  # no two keys equal
    return [
        ("uniform-open-2^18", workloads.uniform(1 << 18, 20), 0.0, 1),
        ("zeldovich-64^3", workloads.zeldovich(64, 3), 1.0, 1),
        ("duplicates-2^17", x_dup, 0.0, 1),
        ("ragged-65536+4093", workloads.uniform(65536 + 4093, 22), 1.0, 1),
        ("dense-blob-big-bin", x_blob, 0.0, 1),
        ("heavy-bin-fallback", x_heavy, 1.0, 0),
    ]


@pytest.mark.parametrize("name,x,L,path", _bucket_cases(), ids=[c[0] for c in _bucket_cases()])
def test_bucket_sort_matches_oracle(name, x, L, path):
    """Sets of 2^16 points and more sort their keys by fine bins and per-group
    shared-memory passes (LSD passes when a bin is too full): the same stable
    order, gathered points and tree as the oracle, bit-exact, and the same
    arrays as a build that forces the LSD passes."""
    import paper_2604_05885_gb300 as jzt
    xt = to_dev(x)
    tree = jzt.build(xt, periodic_L=L)
    st = tree.status()
    assert st["code"] == 0, st
    assert st["sort_path"] == path
    keys, pts, n_planes = tree.arrays()
    keys = keys.cpu().numpy().view(np.uint64)
    p_np = pts.cpu().numpy()
    sk, perm = oracle.zsort(oracle.morton_keys(x, L))
    assert np.array_equal(keys, sk), f"sorted keys differ at {int(np.argmax(keys != sk))}"
    assert np.array_equal(p_np[:, 3].view(np.int32), perm.astype(np.int32)), "sort order"
    assert np.array_equal(p_np[:, :3], x[perm]), "gathered points"
    spl_ref, gaps_ref = oracle.plane_splits(sk, nmax0=32, c=8, n_target=1000)  # library defaults
    nodes_ref = oracle.plane_nodes(x[perm], gaps_ref)
    assert n_planes == len(spl_ref)
    lsd = jzt.build(xt, periodic_L=L, params=dict(lsd_sort=1))
    assert lsd.status()["sort_path"] == 0
    k2, p2, _ = lsd.arrays()
    assert np.array_equal(k2.cpu().numpy().view(np.uint64), keys)
    assert np.array_equal(p2.cpu().numpy().view(np.int32), p_np.view(np.int32))
    for pl in range(n_planes):
        spl, cnt, box = tree.plane(pl)
        assert np.array_equal(spl, spl_ref[pl].astype(np.int32)), f"plane {pl} splits"
        rc, rlo, rhi = nodes_ref[pl]
        assert np.array_equal(cnt, rc.astype(np.int32)), f"plane {pl} counts"
        assert np.array_equal(box[:, :3], rlo) and np.array_equal(box[:, 3:], rhi), f"plane {pl} boxes"
