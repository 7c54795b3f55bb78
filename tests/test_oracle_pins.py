"""Pins of the float64 oracle against what the paper and mathematics fix (closed forms, invariants,
brute force).  CPU only."""
import numpy as np
import pytest
from scipy import integrate

from oracle import affine, mc, mlp, octree
from synth import boxes, fields, inr


@pytest.fixture(scope="module")
def small():
    layers, isos, wl = inr.load_inr("small")
    return layers, isos, wl


def _linear_regime_net(seed, dims, sign):
    """ReLU MLP whose pre-activations keep one sign on [-1,1]^3: with sign=+1 every ReLU is the
    identity (the net is linear), with sign=-1 every hidden ReLU outputs 0 in layer 1."""
    rng = np.random.default_rng(seed)
    layers = []
    m = 1.0                                  # bound on |input| of the current layer
    for l, (a, b) in enumerate(zip(dims[:-1], dims[1:])):
        W = rng.uniform(0.1, 1.0, size=(b, a)) * rng.choice([-1, 1], size=(b, a))
        if l < len(dims) - 2:
            reach = np.abs(W).sum(axis=1) * m
            bias = sign * (reach + 1.0)
            m = float((reach + np.abs(bias)).max())
        else:
            bias = rng.normal(size=b)
        layers.append((W.astype(np.float64), bias.astype(np.float64)))
    return layers


# ---- P1: Eq. 3 is exact through linear maps ------------------------------------------------

def test_single_linear_layer_radius_is_exact():
    rng = np.random.default_rng(0)
    W = rng.normal(size=(1, 3))
    b = rng.normal(size=1)
    lo, hi = boxes.random_boxes(200, 1, -10, -1)
    x0, r = affine.bound([(W, b)], lo, hi, affine.SOUND)
    lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
    h = (hi64 - lo64) / 2
    xc = (hi64 + lo64) / 2
    np.testing.assert_allclose(r, (h * np.abs(W[0])).sum(1), rtol=1e-12, atol=0)
    np.testing.assert_allclose(x0, xc @ W[0] + b[0], rtol=1e-12, atol=1e-14)
    # the exact range of a linear function over a box is [f(xc) - sum h|w|, f(xc) + sum h|w|]:
    # attained at the corner sign(w) * h
    corner = xc + np.sign(W[0])[None, :] * h
    np.testing.assert_allclose(x0 + r, corner @ W[0] + b[0], rtol=1e-12, atol=1e-14)


def test_linear_composition_radius_and_clt_sigma_are_exact():
    layers = _linear_regime_net(3, [3, 7, 5, 1], +1)
    Weff = layers[2][0] @ layers[1][0] @ layers[0][0]           # (1, 3)
    lo, hi = boxes.random_boxes(100, 4, -6, -1)
    h = (hi.astype(np.float64) - lo.astype(np.float64)) / 2
    x0, r = affine.bound(layers, lo, hi, affine.SOUND)
    np.testing.assert_allclose(r, (h * np.abs(Weff[0])).sum(1), rtol=1e-12)
    xc = (hi.astype(np.float64) + lo.astype(np.float64)) / 2
    np.testing.assert_allclose(x0, mlp.mlp_forward(layers, xc), rtol=1e-12)
    # P3 (ii): with uniform inputs the CLT sigma of a linear net is exact: sqrt(sum (h_k w_k)^2 / 3)
    mu, sig = affine.bound(layers, lo, hi, affine.CLT)
    np.testing.assert_allclose(sig, np.sqrt(((h * Weff[0]) ** 2).sum(1) / 3.0), rtol=1e-12)
    np.testing.assert_allclose(mu, x0, rtol=1e-12)


def test_dead_relu_layer_gives_constant_output():
    layers = _linear_regime_net(5, [3, 6, 4, 1], -1)
    lo, hi = boxes.random_boxes(20, 6, -4, -1)
    for mode in (affine.SOUND, affine.CLT):
        x0, s = affine.bound(layers, lo, hi, mode)
        expect = layers[2][0] @ np.maximum(layers[1][1], 0) + layers[2][1]
        if mode == affine.SOUND:
            np.testing.assert_allclose(x0, expect[0], rtol=1e-12)
            assert np.all(s == 0)


# ---- the ReLU linearisations ---------------------------------------------------------------

def test_chebyshev_relu_equioscillates_and_is_minimax():
    rng = np.random.default_rng(7)
    l = -rng.uniform(0.01, 3, 200)
    u = rng.uniform(0.01, 3, 200)
    a, b, g = affine.relu_chebyshev(l, u)
    e = lambda x, a, b: np.maximum(x, 0) - a * x - b
    np.testing.assert_allclose(e(l, a, b), g, rtol=1e-12)
    np.testing.assert_allclose(e(np.zeros_like(l), a, b), -g, rtol=1e-12)
    np.testing.assert_allclose(e(u, a, b), g, rtol=1e-12)
    xs = np.linspace(0, 1, 2001)[None, :] * (u - l)[:, None] + l[:, None]
    err = np.abs(e(xs, a[:, None], b[:, None])).max(1)
    np.testing.assert_allclose(err, g, rtol=1e-12)
    # any perturbed line has a larger maximum error (Chebyshev alternation => optimal)
    # (the error of any line is piecewise linear in x with breakpoints l, 0, u)
    brk = np.stack([l, np.zeros_like(l), u], axis=1)
    for _ in range(20):
        da, db = rng.normal(scale=1e-3, size=2)
        err2 = np.abs(e(brk, (a + da)[:, None], (b + db)[:, None])).max(1)
        assert np.all(err2 >= g - 1e-12)
    # one-signed intervals are exact
    a, b, g = affine.relu_chebyshev(np.array([0.5, -2.0, 0.0]), np.array([2.0, -0.5, 1.0]))
    np.testing.assert_array_equal(a, [1.0, 0.0, 1.0])
    np.testing.assert_array_equal(g, [0.0, 0.0, 0.0])


def _relu_ls_quadrature(mu, sigma):
    pdf = lambda x: np.exp(-0.5 * ((x - mu) / sigma) ** 2) / (sigma * np.sqrt(2 * np.pi))
    lo, hi = mu - 40 * sigma, mu + 40 * sigma
    q = lambda f: integrate.quad(lambda x: f(x) * pdf(x), lo, hi, points=[0.0] if lo < 0 < hi else None,
                                 epsabs=1e-14, epsrel=1e-13, limit=400)[0]
    ey = q(lambda x: max(x, 0.0))
    exy = q(lambda x: x * max(x, 0.0))
    ey2 = q(lambda x: max(x, 0.0) ** 2)
    alpha = (exy - mu * ey) / sigma ** 2          # least squares: Cov(X, Y) / Var(X)
    beta = ey - alpha * mu
    gamma2 = ey2 - ey ** 2 - alpha ** 2 * sigma ** 2
    return alpha, beta, gamma2


@pytest.mark.parametrize("mu,sigma", [(-2.0, 0.7), (-0.3, 1.0), (0.0, 0.5), (0.4, 0.2), (1.5, 0.6),
                                      (3.0, 1.2), (-1e-3, 2e-3)])
def test_table7_relu_matches_gaussian_least_squares_by_quadrature(mu, sigma):
    """P6: the ReLU row of Table VII equals the least-squares fit of Eq. 10 computed by quadrature."""
    a, b, g = affine.relu_least_squares(np.array([mu]), np.array([sigma]))
    qa, qb, qg2 = _relu_ls_quadrature(mu, sigma)
    assert abs(a[0] - qa) <= 1e-9
    assert abs(b[0] - qb) <= 1e-9 * sigma
    assert abs(g[0] ** 2 - qg2) <= 1e-9 * sigma ** 2


def test_table7_relu_moments_match_monte_carlo():
    """P3 (i): the mean alpha mu + beta and std sqrt(alpha^2 sigma^2 + gamma^2) of the linearised
    ReLU output match 10^6 Monte-Carlo samples of ReLU(N(mu, sigma^2)) within 1 % of sigma (and
    within 1 % relative where the moment exceeds 0.1 sigma)."""
    rng = np.random.default_rng(11)
    z = rng.standard_normal(1_000_000)
    sigma = 0.7
    for t in np.linspace(-3, 3, 13):
        mu = t * sigma
        y = np.maximum(mu + sigma * z, 0)
        a, b, g = affine.relu_least_squares(np.array([mu]), np.array([sigma]))
        mean = a[0] * mu + b[0]
        std = np.sqrt(a[0] ** 2 * sigma ** 2 + g[0] ** 2)
        for est, ref in ((mean, y.mean()), (std, y.std())):
            assert abs(est - ref) <= 0.01 * sigma
            if ref > 0.1 * sigma:
                assert abs(est / ref - 1) <= 0.01


def test_sigma_zero_reading():
    a, b, g = affine.relu_least_squares(np.array([2.0, -1.0, 0.0]), np.zeros(3))
    np.testing.assert_array_equal(a, [1.0, 0.0, 0.5])
    np.testing.assert_array_equal(b, [0, 0, 0])
    np.testing.assert_array_equal(g, [0, 0, 0])


# ---- P10: the CLT sigma equals the covariance propagation ------------------------------------

def test_clt_sigma_matches_covariance_propagation(small):
    layers, _, _ = small
    lo, hi = boxes.random_boxes(64, 21, -8, -1)
    mu, sig = affine.bound(layers, lo, hi, affine.CLT)
    mu2, sig2 = affine.clt_covariance(layers, lo, hi)
    np.testing.assert_allclose(mu, mu2, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(sig, sig2, rtol=1e-12)
    deep = inr.random_inr([3, 16, 16, 16, 1], 4)
    mu, sig = affine.bound(deep, lo, hi, affine.CLT)
    mu2, sig2 = affine.clt_covariance(deep, lo, hi)
    np.testing.assert_allclose(sig, sig2, rtol=1e-12)


# ---- P2: sound bounds contain brute-force samples --------------------------------------------

def test_sound_bounds_contain_samples(small):
    layers, _, _ = small
    rng = np.random.default_rng(5)
    n_box, n_pts = 1000, 10_000
    lo, hi = boxes.random_boxes(n_box, 9, -10, -1)
    x0, r = affine.bound(layers, lo, hi, affine.SOUND, batch=256)
    lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
    corners = np.array([[(c >> d) & 1 for d in range(3)] for c in range(8)], dtype=np.float64)
    faces = np.array([[0.5, 0.5, 0.0], [0.5, 0.5, 1.0], [0.5, 0.0, 0.5], [0.5, 1.0, 0.5],
                      [0.0, 0.5, 0.5], [1.0, 0.5, 0.5]])
    worst = -np.inf
    for s in range(0, n_box, 50):
        sl = slice(s, s + 50)
        u = np.concatenate([rng.uniform(size=(50, n_pts, 3)), np.broadcast_to(corners, (50, 8, 3)),
                            np.broadcast_to(faces, (50, 6, 3))], axis=1)
        pts = lo64[sl, None, :] + u * (hi64 - lo64)[sl, None, :]
        v = mlp.mlp_forward(layers, pts.reshape(-1, 3)).reshape(50, -1)
        excess = np.maximum(v.max(1) - (x0[sl] + r[sl]), (x0[sl] - r[sl]) - v.min(1))
        worst = max(worst, excess.max())
    assert worst <= 1e-12        # float64 rounding of the oracle itself


# ---- P4 / P7 / P8: hierarchy against the dense truth ----------------------------------------

def test_sound_hierarchy_matches_dense_marching_cubes(small):
    """P4: sound-bound extraction gives exactly the dense marching-cubes triangle set."""
    layers, isos, wl = small
    R = 1 << wl.max_level
    vals = mlp.mlp_forward(layers, octree.lattice_points(R))
    levels = octree.extract_active(layers, wl.max_level, isos, affine.SOUND, batch=512)
    act, _ = octree.active_cells(levels)
    dense_cells = mc.crossing_cells(vals, R, isos[0])
    e_h, _, _ = mc.march(vals, act, R, isos[0])
    e_d, _, _ = mc.march(vals, dense_cells, R, isos[0])
    assert e_d.shape[0] > 1000
    np.testing.assert_array_equal(mc.sorted_edge_triples(e_h), mc.sorted_edge_triples(e_d))


def test_brute_force_8cubed_sound_and_clt_infinite_k():
    """P7: at 8^3 sound bounds (and CLT with k = inf) never miss a dense crossing cell."""
    layers = inr.random_inr([3, 24, 24, 1], 13)
    R, L = 8, 3
    vals = mlp.mlp_forward(layers, octree.lattice_points(R))
    isos = np.quantile(vals, [0.3, 0.5, 0.7])
    for mode, k in ((affine.SOUND, 0.0), (affine.CLT, np.inf)):
        levels = octree.extract_active(layers, L, isos, mode, k=k)
        act, mask = octree.active_cells(levels)
        for q, c in enumerate(isos):
            truth = mc.crossing_cells(vals, R, c)
            pred = act[(mask >> q) & 1 == 1]
            fpr, fnr = octree.fpr_fnr(pred, truth, R)
            assert fnr == 0.0
    levels = octree.extract_active(layers, L, isos, affine.CLT, k=np.inf)
    assert all(np.all(lv["mask"] == lv["mask_in"]) for lv in levels)


def test_clt_active_sets_grow_with_k(small):
    """P8: (mu, sigma) do not depend on k, so active sets are nested in k at every level."""
    layers, isos, wl = small
    sets = []
    for k in (2.0, 3.0, 4.0):
        levels = octree.extract_active(layers, 4, isos, affine.CLT, k=k, batch=512)
        sets.append([set(map(tuple, lv["ijk"][lv["mask"] != 0])) for lv in levels])
    for a, b in zip(sets[:-1], sets[1:]):
        for la, lb in zip(a, b):
            assert la <= lb


# ---- marching cubes ------------------------------------------------------------------------

def _mesh_stats(edges, verts):
    ids, inv = np.unique(edges.ravel(), return_inverse=True)
    tri = inv.reshape(-1, 3)
    und = np.sort(np.stack([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], 1).reshape(-1, 2), axis=1)
    ue, cnt = np.unique(und, axis=0, return_counts=True)
    directed = np.stack([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]], 1).reshape(-1, 2)
    from collections import Counter
    dcnt = Counter(map(tuple, directed.tolist()))
    # closed and consistently oriented: every directed edge is matched by as many reversed ones
    opposite_ok = all(dcnt[(b, a)] == n for (a, b), n in dcnt.items())
    opposite_ok = opposite_ok and bool(np.all((tri[:, 0] != tri[:, 1]) & (tri[:, 1] != tri[:, 2])
                                              & (tri[:, 0] != tri[:, 2])))
    V, E, F = ids.size, ue.shape[0], tri.shape[0]
    parent = np.arange(V)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for a, b in ue:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
    comps = len({find(i) for i in range(V)})
    p = verts
    area = 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1).sum()
    vol = np.einsum("ti,ti->t", p[:, 0], np.cross(p[:, 1], p[:, 2])).sum() / 6.0
    return dict(V=V, E=E, F=F, chi=V - E + F, max_share=cnt.max(), min_share=cnt.min(),
                opposite_ok=opposite_ok, comps=comps, area=area, vol=vol)


@pytest.mark.parametrize("R", [64, 128])
def test_sphere_mesh(R):
    """P5: marching cubes on |x| - 0.5 gives a closed, consistently oriented genus-0 sphere."""
    rad = 0.5
    vals = fields.sphere_sdf(rad)(octree.lattice_points(R))
    cells = mc.crossing_cells(vals, R, 0.0)
    e, p, _ = mc.march(vals, cells, R, 0.0)
    st = _mesh_stats(e, p)
    assert st["max_share"] == 2 and st["min_share"] == 2 and st["opposite_ok"]
    assert st["chi"] == 2 and st["comps"] == 1
    h = 2.0 / R
    assert np.abs(np.linalg.norm(p.reshape(-1, 3), axis=1) - rad).max() <= h * h / (4 * rad)
    assert abs(st["area"] / (4 * np.pi * rad ** 2) - 1) < 0.01
    assert abs(st["vol"] / (4 / 3 * np.pi * rad ** 3) - 1) < 0.01
    # normals point toward increasing values (outward)
    n = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    assert np.all(np.einsum("ti,ti->t", n, p.mean(1)) > 0)


def test_sphere_volume_converges_quadratically():
    errs = []
    for R in (32, 64, 128):
        vals = fields.sphere_sdf(0.5)(octree.lattice_points(R))
        e, p, _ = mc.march(vals, mc.crossing_cells(vals, R, 0.0), R, 0.0)
        errs.append(abs(_mesh_stats(e, p)["vol"] / (4 / 3 * np.pi * 0.125) - 1))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_marching_cubes_vertices_lie_on_planes():
    """Linear interpolation is exact for a linear field: every vertex lies on the plane."""
    R = 16
    rng = np.random.default_rng(2)
    for _ in range(5):
        a = rng.normal(size=3)
        d = rng.normal() * 0.3
        pts = octree.lattice_points(R)
        vals = pts @ a + d
        e, p, _ = mc.march(vals, mc.crossing_cells(vals, R, 0.0), R, 0.0)
        assert np.abs(p.reshape(-1, 3) @ a + d).max() < 1e-12
        n = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
        assert np.all(n @ a > 0)


def test_marching_cubes_random_fields_are_watertight():
    """Every interior edge of the mesh of a random lattice field is shared by exactly two
    triangles with opposite directions (covers the ambiguous-face rule on all 256 cases)."""
    rng = np.random.default_rng(3)
    R = 12
    seen = set()
    for _ in range(6):
        vals = rng.normal(size=(R + 1) ** 3)
        # pad a boundary layer of +1 (outside) so that every surface is closed
        v3 = vals.reshape(R + 1, R + 1, R + 1)
        v3[[0, -1], :, :] = 1.0
        v3[:, [0, -1], :] = 1.0
        v3[:, :, [0, -1]] = 1.0
        cells = mc.crossing_cells(v3.ravel(), R, 0.0)
        seen.update(mc.cell_cases(mc.corner_values(v3.ravel(), cells, R), 0.0).tolist())
        e, p, _ = mc.march(v3.ravel(), cells, R, 0.0)
        st = _mesh_stats(e, p)
        # a loop that meets a face twice can put a fan diagonal in the face plane, where the
        # neighbour's diagonal meets it: such edges are shared by 4 triangles (still closed)
        assert st["min_share"] == 2 and st["max_share"] % 2 == 0 and st["opposite_ok"]
    assert len(seen) > 200


def test_mc_table_matches_golden():
    """The committed table (written by tests/golden/make_golden.py from this oracle) is current."""
    import os
    ntri, tab = mc.build_table()
    path = os.path.join(os.path.dirname(__file__), "golden", "mc_table.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 256
    for c, r in enumerate(rows):
        vals = list(map(int, r))
        assert vals[0] == c and vals[1] == ntri[c]
        assert vals[2:] == tab[c].ravel().tolist()


def test_kd_tree_leaves_are_octree_cubes_and_nested():
    """Algorithm 1's k-d tree bounds every octree cube and the two intermediate boxes between
    consecutive cube depths, so its leaves at depth 3 L are a subset of the octree's active cells
    (same mode and k), and sound bounds still never miss a dense crossing cell (brute force, 8^3)."""
    layers = inr.random_inr([3, 16, 16, 1], 5)
    L = 3
    vals = mlp.mlp_forward(layers, octree.lattice_points(1 << L))
    isos = np.quantile(vals, [0.3, 0.7])
    for mode, k in (("sound", 0.0), ("clt", 2.0)):
        kd = octree.kd_extract_active(layers, L, isos, mode, k=k, batch=64)
        oc = octree.extract_active(layers, L, isos, mode, k=k, batch=64)
        kd_cells, kd_masks = octree.active_cells(kd)
        oc_cells, oc_masks = octree.active_cells(oc)
        occ = {tuple(c): m for c, m in zip(oc_cells.tolist(), oc_masks.tolist())}
        for c, m in zip(kd_cells.tolist(), kd_masks.tolist()):
            assert tuple(c) in occ and (m & ~occ[tuple(c)]) == 0
        # every third depth holds cubes: their boxes equal the octree's boxes of that level
        for d in (0, 3, 6):
            lo, hi = octree.kd_box(kd[d]["ijk"], d)
            lo2, hi2 = octree.cell_box(kd[d]["ijk"], d // 3)
            assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)
        if mode == "sound":
            got = {tuple(c): m for c, m in zip(kd_cells.tolist(), kd_masks.tolist())}
            for q, iso in enumerate(isos):
                for c in mc.crossing_cells(vals, 1 << L, iso).tolist():
                    assert tuple(c) in got and (got[tuple(c)] >> q) & 1


# ---- RA-Fixed: the reduced form against full affine arithmetic and brute force ----------------

def test_rafixed_one_hidden_layer_equals_full_affine():
    """With one hidden layer the only condensed symbols are the ReLU's own, whose output
    coefficients w_m gamma_m add up in absolute value to |w| gamma either way: RA-Fixed and full
    affine arithmetic give the same centre and radius."""
    layers = inr.random_inr([3, 48, 1], 11)
    lo, hi = boxes.random_boxes(200, 3, -6, -1)
    c0, r0 = affine.bound(layers, lo, hi, affine.SOUND)
    c1, r1 = affine.bound(layers, lo, hi, affine.RAFIXED)
    assert np.allclose(c0, c1, rtol=1e-12, atol=1e-12) and np.allclose(r0, r1, rtol=1e-12, atol=1e-12)


def test_rafixed_two_hidden_layers_is_full_affine_loosened():
    """With two hidden layers the second layer's pre-activation radius is the same (sum_m |W_nm|
    gamma_m either way), so the second ReLU's lines and the centre agree; at the output the
    condensed radius sum_n |w_n| alpha_n |W_nm| gamma_m bounds the full form's |sum_n ...| term by
    term: RA-Fixed radius >= full radius, with a strict gap for most boxes."""
    layers = inr.random_inr([3, 32, 32, 1], 12)
    lo, hi = boxes.random_boxes(300, 4, -5, -1)
    c0, r0 = affine.bound(layers, lo, hi, affine.SOUND)
    c1, r1 = affine.bound(layers, lo, hi, affine.RAFIXED)
    assert np.allclose(c0, c1, rtol=1e-11, atol=1e-12)
    assert np.all(r1 >= r0 - 1e-12 * np.abs(r0))
    assert np.mean(r1 > r0 * (1 + 1e-9)) > 0.5


def test_rafixed_bounds_contain_samples_and_linear_nets_are_exact(small):
    layers, _, _ = small
    rng = np.random.default_rng(6)
    lo, hi = boxes.random_boxes(400, 10, -8, -1)
    c, r = affine.bound(layers, lo, hi, affine.RAFIXED, batch=200)
    lo64, hi64 = lo.astype(np.float64), hi.astype(np.float64)
    u = rng.uniform(size=(400, 2000, 3))
    corners = np.array([[(q >> d) & 1 for d in range(3)] for q in range(8)], dtype=np.float64)
    u = np.concatenate([u, np.broadcast_to(corners, (400, 8, 3))], axis=1)
    pts = lo64[:, None, :] + u * (hi64 - lo64)[:, None, :]
    v = mlp.mlp_forward(layers, pts.reshape(-1, 3)).reshape(400, -1)
    assert np.all(v.max(1) <= c + r + 1e-12) and np.all(v.min(1) >= c - r - 1e-12)
    # a net whose ReLUs are all the identity on [-1, 1]^3 is affine: the radius is exact
    lin = _linear_regime_net(7, [3, 8, 8, 8, 1], +1)
    lo, hi = boxes.random_boxes(50, 8, -4, -1)
    c, r = affine.bound(lin, lo, hi, affine.RAFIXED)
    Weff = lin[0][0]
    for W, _ in lin[1:]:
        Weff = W @ Weff
    h = (hi.astype(np.float64) - lo.astype(np.float64)) / 2
    assert np.allclose(r, np.abs(Weff[0]) @ h.T, rtol=1e-10)


# ---- ELU and sine activations: least-squares lines against Table VII and quadrature ------------

from oracle import activations as acts  # noqa: E402
from scipy.special import erf  # noqa: E402

_GRID = [(mu, sg) for mu in (-4.0, -1.3, -0.2, 0.0, 0.4, 2.5) for sg in (0.05, 0.4, 1.0, 2.2)]


def _table7_sine(mu, sg):
    """Table VII, sine row, as printed."""
    a = np.exp(-0.5 * sg ** 2)
    alpha = a * np.cos(mu)
    beta = a * (np.sin(mu) - mu * np.cos(mu))
    g2 = -a ** 2 * (sg ** 2 * np.cos(mu) ** 2 + np.sin(mu) ** 2) + 0.5 * (1 - a ** 4 * np.cos(2 * mu))
    return alpha, beta, g2


def _table7_elu(mu, sg):
    """Table VII, ELU row, as printed."""
    a = erf(-mu / (np.sqrt(2) * sg))
    b = (1 + erf((-mu - sg ** 2) / (np.sqrt(2) * sg))) * np.exp(mu + sg ** 2 / 2)
    alpha = 0.5 * (1 - a + b)
    c = np.exp(-mu ** 2 / (2 * sg ** 2)) / np.sqrt(2 * np.pi)
    beta = 0.5 * b * (1 - mu) - 0.5 * (1 + a) + c * sg
    g2 = (0.25 * (1 - a ** 2) * (mu ** 2 + sg ** 2) + (0.5 * a * b - c ** 2 - 0.25 * b ** 2 - 0.5 * b) * sg ** 2
          + a * c * mu * sg + (a - b + 1) * c * sg + 0.5 * (a * b - b - a ** 2 + 1) * mu
          + 0.25 * (1 + erf((-mu - 2 * sg ** 2) / (np.sqrt(2) * sg))) * np.exp(2 * mu + 2 * sg ** 2)
          + 0.25 - 0.25 * (a - b) ** 2 - 0.5 * b)
    return alpha, beta, g2


@pytest.mark.parametrize("act", [acts.SINE, acts.ELU])
def test_table7_sine_and_elu_rows(act):
    """The moments-based fit equals Table VII's printed closed forms: alpha, beta and gamma^2 of the
    sine row, alpha and beta of the ELU row.  The ELU row's gamma^2 as printed is negative over most
    of the grid (e.g. -0.23 at mu = 0, sigma = 0.05), so it cannot be the residual variance; gamma^2
    is taken from its definition and pinned by quadrature (test below)."""
    table = _table7_sine if act == acts.SINE else _table7_elu
    for mu, sg in _GRID:
        al, be, ga = acts.least_squares(act, mu, sg)
        ta, tb, tg2 = table(mu, sg)
        scale = max(1.0, mu * mu + sg * sg)
        assert abs(al - ta) <= 1e-12 * max(1, abs(ta)), (act, mu, sg)
        assert abs(be - tb) <= 1e-12 * max(1, abs(tb)), (act, mu, sg)
        if act == acts.SINE:
            assert abs(ga ** 2 - max(tg2, 0.0)) <= 1e-12 * scale, (act, mu, sg, ga ** 2, tg2)
    if act == acts.ELU:
        assert _table7_elu(0.0, 0.05)[2] < -0.2 and acts.least_squares(acts.ELU, 0.0, 0.05)[2] > 0


@pytest.mark.parametrize("act", [acts.RELU, acts.SINE, acts.ELU])
def test_least_squares_fit_by_quadrature(act):
    """Normal equations E[r] = E[r X] = 0 and gamma^2 = E[r^2] for the residual r = f(X) - alpha X - beta,
    X ~ N(mu, sigma^2), by numerical integration; the ReLU row also equals affine.relu_least_squares."""
    for mu, sg in _GRID:
        al, be, ga = acts.least_squares(act, mu, sg)

        def dens(x):
            return np.exp(-0.5 * ((x - mu) / sg) ** 2) / (np.sqrt(2 * np.pi) * sg)

        def r(x):
            return float(acts.forward(act, x)) - al * x - be

        lo, hi = mu - 12 * sg, mu + 12 * sg
        pts = [0.0] if lo < 0 < hi else None
        e0 = integrate.quad(lambda x: r(x) * dens(x), lo, hi, points=pts, limit=400, epsabs=1e-13)[0]
        e1 = integrate.quad(lambda x: r(x) * (x - mu) * dens(x), lo, hi, points=pts, limit=400, epsabs=1e-13)[0]
        e2 = integrate.quad(lambda x: r(x) ** 2 * dens(x), lo, hi, points=pts, limit=400, epsabs=1e-13)[0]
        scale = max(1.0, abs(mu) + sg)
        assert abs(e0) <= 1e-8 * scale and abs(e1) <= 1e-8 * scale * sg, (act, mu, sg, e0, e1)
        assert abs(e2 - ga ** 2) <= 1e-8 * scale ** 2, (act, mu, sg, e2, ga ** 2)
        if act == acts.RELU:
            ra, rb, rg = affine.relu_least_squares(mu, sg)
            assert abs(al - ra) <= 1e-12 and abs(be - rb) <= 1e-12 * scale
            assert abs(ga ** 2 - rg ** 2) <= 1e-13 * scale ** 2


@pytest.mark.parametrize("act", [acts.SINE, acts.ELU, acts.RELU])
def test_least_squares_small_sigma_is_the_tangent(act):
    for mu in (-2.0, -0.5, 0.3, 1.7):
        al, be, ga = acts.least_squares(act, mu, 1e-4)
        t_al, t_be, t_ga = acts.least_squares(act, mu, 0.0)
        assert abs(al - t_al) < 1e-7 and abs(be - t_be) < 1e-7 and t_ga == 0 and ga < 1e-7


def test_relu_least_squares_at_the_kink_is_continuous_in_sigma():
    """At mu = 0 the ReLU row gives alpha = P(X > 0) = 1/2 for every sigma > 0, so the sigma = 0
    reading (alpha = 1/2 at mu = 0) is the limit; both ReLU rules agree there."""
    for sg in (1.0, 1e-3, 1e-12):
        assert acts.least_squares(acts.RELU, 0.0, sg)[0] == pytest.approx(0.5, abs=1e-15)
    al, be, ga = acts.least_squares(acts.RELU, 0.0, 0.0)
    assert (al, be, ga) == (0.5, 0.0, 0.0)
    a2 = affine.relu_least_squares(np.array([0.0]), np.array([0.0]))
    assert (a2[0][0], a2[1][0], a2[2][0]) == (0.5, 0.0, 0.0)


def test_canonical_triangle_form_keeps_orientation():
    """A triangle (a, b, c) is the same oriented triangle as (b, c, a) and (c, a, b), not as
    (a, c, b): the canonical form rotates each triple to its smallest id and sorts the rows."""
    got = mc.sorted_edge_triples([[9, 3, 5], [7, 8, 6], [2, 1, 4]])
    np.testing.assert_array_equal(got, [[1, 4, 2], [3, 5, 9], [6, 7, 8]])
    assert not np.array_equal(mc.sorted_edge_triples([[1, 2, 3]]), mc.sorted_edge_triples([[1, 3, 2]]))


@pytest.mark.parametrize("act", [acts.SINE, acts.ELU])
def test_up_mean_of_one_hidden_layer_equals_gaussian_input_expectation(act):
    """With one hidden layer the propagated mean is b_out + sum_n w_n E f(z_n), z_n ~ N(mu_n,
    sigma_n^2) from the Gaussian reading of the input box: it equals the Monte Carlo mean of the network
    driven by x ~ N(x_c, diag(h^2 / 3)), whose pre-activations are exactly those Gaussians."""
    layers = inr.random_inr([3, 24, 1], 19)
    if act == acts.SINE:
        layers = [(W * 6.0, b * 6.0) for W, b in layers[:1]] + layers[1:]
    rng = np.random.default_rng(20)
    lo, hi = np.array([[-0.4, 0.1, -0.3]]), np.array([[0.2, 0.5, 0.1]])
    mu, _ = affine.bound(layers, lo, hi, affine.CLT, act=act)
    xc, h = (lo + hi)[0] / 2, (hi - lo)[0] / 2
    x = xc + rng.normal(size=(2_000_000, 3)) * h / np.sqrt(3)
    v = mlp.mlp_forward(layers, x, act=act)
    assert abs(mu[0] - v.mean()) <= 5 * v.std() / np.sqrt(x.shape[0])


def test_raua_readout_exact_on_linear_nets_and_inside_the_sound_radius(small):
    """RA-UA (Sec. IV-A): sound propagation read off with sigma^2 = (1/3) sum x_i^2.  On a net that is
    affine over the domain this is the exact standard deviation of the output under uniform inputs;
    on any net sqrt(3) sigma = ||x||_2 <= ||x||_1 = the sound radius, with the sound centre."""
    layers = _linear_regime_net(3, [3, 7, 5, 1], +1)
    Weff = layers[2][0] @ layers[1][0] @ layers[0][0]
    lo, hi = boxes.random_boxes(100, 4, -6, -1)
    h = (hi.astype(np.float64) - lo.astype(np.float64)) / 2
    c, sig = affine.bound(layers, lo, hi, affine.RAUA)
    np.testing.assert_allclose(sig, np.sqrt(((h * Weff[0]) ** 2).sum(1) / 3.0), rtol=1e-12)
    layers, _, _ = small
    lo, hi = boxes.random_boxes(300, 5, -8, -1)
    c, sig = affine.bound(layers, lo, hi, affine.RAUA)
    c0, r0 = affine.bound(layers, lo, hi, affine.SOUND)
    np.testing.assert_allclose(c, c0, rtol=1e-12, atol=1e-15)
    assert np.all(np.sqrt(3.0) * sig <= r0 * (1 + 1e-12))
    assert np.mean(np.sqrt(3.0) * sig < 0.9 * r0) > 0.5          # strictly tighter on most boxes


def test_brute_force_8cubed_rafixed_and_kd_never_miss():
    """RA-Fixed is sound: at 8^3 its hierarchical extraction keeps every dense crossing cell, in the
    octree and in the k-d tree; and on a one-hidden-layer net, where its bound equals full affine
    arithmetic's box by box, both give the same active set."""
    layers = inr.random_inr([3, 24, 24, 1], 14)
    R, L = 8, 3
    vals = mlp.mlp_forward(layers, octree.lattice_points(R))
    isos = np.quantile(vals, [0.3, 0.6])
    for levels in (octree.extract_active(layers, L, isos, affine.RAFIXED),
                   octree.kd_extract_active(layers, L, isos, affine.RAFIXED)):
        act, mask = octree.active_cells(levels)
        for q, c in enumerate(isos):
            truth = mc.crossing_cells(vals, R, c)
            fpr, fnr = octree.fpr_fnr(act[(mask >> q) & 1 == 1], truth, R)
            assert fnr == 0.0
    one = inr.random_inr([3, 32, 1], 15)
    v1 = mlp.mlp_forward(one, octree.lattice_points(R))
    iso1 = np.quantile(v1, [0.5])
    a_fix = octree.active_cells(octree.extract_active(one, L, iso1, affine.RAFIXED))[0]
    a_aa = octree.active_cells(octree.extract_active(one, L, iso1, affine.SOUND))[0]
    assert set(map(tuple, a_fix.tolist())) == set(map(tuple, a_aa.tolist()))


# ---- Worked by hand: a 3 -> 2 -> 2 -> 1 net on the box [-1, 1]^3 -----------------------------

def _hand_net():
    """f(x, y, z) = relu(relu x + relu y) + relu(relu x - relu y): W0 picks x and y, W1 = [[1, 1],
    [1, -1]], W2 = [1, 1], all biases 0.  Its range on [-1, 1]^3 is [0, 2]."""
    return [(np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]), np.zeros(2)),
            (np.array([[1.0, 1.0], [1.0, -1.0]]), np.zeros(2)),
            (np.array([[1.0, 1.0]]), np.zeros(1))]


def test_hand_worked_affine_and_rafixed_bounds():
    """Eq. 3 and Eq. 4 (Chebyshev line) carried out by hand on [-1, 1]^3:
    layer 0: both neurons are the input symbols x, y on [-1, 1]; ReLU: alpha = 1/2, beta = gamma =
    1/4, so each neuron is 1/4 + x/2 + e/4 with its own new symbol e.
    layer 1: neuron 1 = 1/2 + (x + y)/2 + (e1 + e2)/4, neuron 2 = (x - y)/2 + (e1 - e2)/4, each of
    radius 3/2.  ReLU on [-1, 2]: alpha = 2/3, beta = gamma = 1/3; on [-3/2, 3/2]: alpha = 1/2,
    beta = gamma = 3/8.
    output: centre 2/3 + 3/8 = 25/24; coefficients x 7/12, y 1/12, e1 7/24, e2 1/24, e3 1/3, e4 3/8,
    radius 41/24.
    RA-Fixed keeps x, y and gives each neuron a private radius: 1/4 after ReLU 1, |W1| (1/4, 1/4) =
    (1/2, 1/2) after layer 1 (e1, e2 no longer cancel), alpha r + gamma = (2/3, 5/8) after ReLU 2,
    so the output radius is 7/12 + 1/12 + 2/3 + 5/8 = 47/24 about the same centre."""
    L = _hand_net()
    lo, hi = np.full((1, 3), -1.0), np.full((1, 3), 1.0)
    c, r = affine.bound(L, lo, hi, affine.SOUND)
    assert c[0] == pytest.approx(25 / 24, abs=1e-15) and r[0] == pytest.approx(41 / 24, abs=1e-15)
    c, r = affine.bound(L, lo, hi, affine.RAFIXED)
    assert c[0] == pytest.approx(25 / 24, abs=1e-15) and r[0] == pytest.approx(47 / 24, abs=1e-15)
    # both contain the true range [0, 2]
    assert 25 / 24 - 41 / 24 <= 0.0 and 25 / 24 + 41 / 24 >= 2.0


# ---- The cull test is closed at both ends, and culled iso-values stay culled -------------------

def test_plane_on_cell_faces_keeps_both_neighbouring_columns():
    """f(x) = relu(x + 1) - 1 = x on [-1, 1]^3 (the ReLU sees only non-negative inputs, so its line
    is the identity and the sound bound of a cell is exactly [lo_x, hi_x]).  The iso-value 0 lies
    on the faces x = 0 between the columns i = R/2 - 1 and i = R/2: both touch it at a bound
    endpoint and, with the cull test strict (keep on equality), both are active -- 2 R^2 cells."""
    L = [(np.array([[1.0, 0.0, 0.0]]), np.array([1.0])), (np.array([[1.0]]), np.array([-1.0]))]
    for lev in (1, 2, 3):
        R = 1 << lev
        act, _ = octree.active_cells(octree.extract_active(L, lev, [0.0], affine.SOUND))
        assert act.shape[0] == 2 * R * R
        assert set(np.unique(act[:, 0]).tolist()) == {R // 2 - 1, R // 2}


def test_iso_sets_shrink_down_the_tree(small):
    """A child inherits the iso set that survived its parent's test (Algorithm 1 recurses only
    into the parent's surviving iso-values), so every level's incoming set is its parent's
    surviving set, and a surviving set is a subset of the incoming one."""
    layers, isos, _ = small
    lv = octree.extract_active(layers, 4, np.quantile(mlp.mlp_forward(layers, octree.lattice_points(16)),
                                                       [0.2, 0.5, 0.8]), affine.SOUND)
    shrank = 0
    for a, b in zip(lv[:-1], lv[1:]):
        keep = a["mask"] != 0
        parent_mask = a["mask"][keep]
        assert np.array_equal(b["mask_in"], np.repeat(parent_mask, 8))
        assert np.all((b["mask"] & ~b["mask_in"]) == 0)
        shrank += int(np.sum(a["mask"][keep] != a["mask_in"][keep]))
    assert shrank > 0                     # some cell dropped one iso-value but kept another


def test_fpr_fnr_counts():
    """FPR = FP / (FP + TN), FNR = FN / (FN + TP) over the R^3 cells (Sec. V-A.3).  R = 2: truth
    {(0,0,0), (1,0,0)}, prediction {(1,0,0), (0,1,0), (1,1,0)}: TP 1, FP 2, FN 1, TN 4."""
    fpr, fnr = octree.fpr_fnr([[1, 0, 0], [0, 1, 0], [1, 1, 0]], [[0, 0, 0], [1, 0, 0]], 2)
    assert fpr == pytest.approx(2 / 6) and fnr == pytest.approx(1 / 2)
    assert octree.fpr_fnr([[0, 0, 0]], [[0, 0, 0]], 2) == (0.0, 0.0)
    assert octree.fpr_fnr(np.zeros((0, 3)), [[1, 1, 1]], 2) == (0.0, 1.0)
