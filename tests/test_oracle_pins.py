"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test ties one oracle function to something other than itself: a closed
form, a brute-force definition written independently here, a library routine
(scipy's Dijkstra and periodic k-d tree), an analytic law, or a number the
paper prints (tests/golden/paper_constants.json).  No GPU needed.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import dijkstra
from scipy.spatial import cKDTree

from paper_1701_06658_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


# ---------------------------------------------------------------- predictor

def test_taps_are_the_heat_kernel(oracle):
    """Eq. (7)-(9): the taps are a normalised, symmetric Gaussian whose
    variance is 2 dt (the heat kernel at time dt), not dt or 2 pi."""
    for dt in (0.5, 0.75, 1.0):
        g = oracle.heat_kernel_taps(dt, 5)
        k = np.arange(-5, 6)
        assert abs(g.sum() - 1.0) < 1e-15
        assert np.allclose(g, g[::-1], rtol=0, atol=0)
        var = float((g * k * k).sum())
        assert abs(var - 2.0 * dt) / (2.0 * dt) < 2e-3, (dt, var)
        # successive ratios of a sampled Gaussian: g[k+1]/g[k] = exp(-(2k+1)/(4 dt))
        assert abs(g[6] / g[5] - math.exp(-1.0 / (4.0 * dt))) < 1e-14


def _direct_conv(phi, full, taps, eps):
    """Brute-force triple sum over the (2R+1)^3 stencil with explicit lookups."""
    R = (len(taps) - 1) // 2
    nz, ny, nx = phi.shape
    out = np.zeros_like(phi)
    axes3 = [nz > 1 or full[0], True, True]
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        acc = 0.0
        for kz in (range(-R, R + 1) if nz > 1 else [0]):
            for ky in range(-R, R + 1):
                for kx in range(-R, R + 1):
                    p = [z + kz, y + ky, x + kx]
                    n = [nz, ny, nx]
                    val = None
                    for a in range(3):
                        if 0 <= p[a] < n[a]:
                            continue
                        if full[a]:
                            p[a] %= n[a]
                        else:
                            val = -eps
                    if val is None:
                        val = phi[p[0], p[1], p[2]]
                    wz = taps[kz + R] if nz > 1 else 1.0
                    acc += wz * taps[ky + R] * taps[kx + R] * val
        out[z, y, x] = acc
    assert axes3
    return out


@pytest.mark.parametrize("full", [(False, False, False), (True, False, True)])
def test_convolution_equals_direct_sum(oracle, full):
    rng = np.random.default_rng(3)
    phi = rng.uniform(-7, 7, size=(4, 5, 6))
    taps = oracle.heat_kernel_taps(0.7, 2)
    got = oracle.convolve(phi, full, taps, 7.0, (0, 1, 2))
    ref = _direct_conv(phi, full, taps, 7.0)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_convolution_2d_equals_direct_sum(oracle):
    rng = np.random.default_rng(4)
    phi = rng.uniform(-7, 7, size=(1, 6, 7))
    taps = oracle.heat_kernel_taps(1.0, 3)
    got = oracle.convolve(phi, (True, False, False), taps, 7.0, (1, 2))
    ref = _direct_conv(phi, (True, False, False), taps, 7.0)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_convolution_keeps_linear_and_heats_quadratic(oracle):
    """A symmetric normalised kernel leaves linear functions unchanged; on a
    paraboloid |x|^2 one step adds dt * Laplacian = 2 D dt (heat flow, Eq. (7))."""
    n = 24
    z, y, x = np.meshgrid(*(np.arange(n, dtype=float),) * 3, indexing="ij")
    taps = oracle.heat_kernel_taps(1.0, 5)
    inner = (slice(5, -5),) * 3
    lin = 0.3 * x - 0.2 * y + 0.1 * z + 1.5
    c = oracle.convolve(lin, (False,) * 3, taps, 7.0, (0, 1, 2))
    assert np.max(np.abs(c[inner] - lin[inner])) < 1e-12
    quad = (x - 11.5) ** 2 + (y - 12.0) ** 2 + (z - 11.0) ** 2
    c = oracle.convolve(quad, (False,) * 3, taps, 7.0, (0, 1, 2))
    rise = (c - quad)[inner]
    assert abs(rise.mean() - 6.0) / 6.0 < 3e-3
    assert rise.std() < 1e-10


def test_predictor_moves_exact_sphere_by_curvature(oracle):
    """One predictor step on an exact SDF moves the zero level as motion by
    mean curvature for time dt: r^2 drops by 2 (D-1) dt (Eq. (9))."""
    for dim, n, r in ((2, 96, 20.0), (3, 48, 14.0)):
        c = n / 2.0
        shape = (1, n, n) if dim == 2 else (n, n, n)
        z, y, x = np.meshgrid(*(np.arange(s, dtype=float) for s in shape), indexing="ij")
        rho2 = (x - c) ** 2 + (y - c) ** 2 + (0 if dim == 2 else (z - c) ** 2)
        d = np.clip(r - np.sqrt(rho2), -7, 7)
        axes = oracle.spatial_axes(shape)
        cv = oracle.convolve(d, (True,) * 3, oracle.heat_kernel_taps(1.0, 5), 7.0, axes)
        zc = int(c) if dim == 3 else 0
        row = cv[zc, int(c), :]
        i = next(i for i in range(int(c), n - 1) if row[i] > 0 >= row[i + 1])
        xr = i + row[i] / (row[i] - row[i + 1]) - c
        assert abs((xr * xr - r * r) - (-2.0 * (dim - 1))) < 0.03 * 2 * (dim - 1), (dim, xr * xr - r * r)


# ---------------------------------------------------------------- corrector

def _random_grains(oracle, shape, count, seed):
    rng = np.random.default_rng(seed)
    grains = []
    for g in range(count):
        dims = tuple(int(rng.integers(2, s + 1)) if s > 1 else 1 for s in shape)
        origin = tuple(int(rng.integers(0, s)) for s in shape)
        grains.append(oracle.Grain(g, origin, rng.uniform(-7, 7, size=dims)))
    return grains


def test_neighbour_max_is_literal_max(oracle):
    """Eq. (16)'s max over all other grains, written on dense domain arrays
    (-eps where a box does not reach), equals the box-local computation with
    and without the neighbour preselection; ties go to the lowest id."""
    shape = (5, 6, 7)
    grains = _random_grains(oracle, shape, 6, 11)
    # force exact ties between grains 1 and 4 where both cover the cell
    phip = {g.gid: g.phi.copy() for g in grains}
    dense = np.full((len(grains),) + shape, -7.0)
    allpos = tuple(np.arange(s) for s in shape)
    for g in grains:
        v, mask = oracle.sample(g, allpos, shape, -7.0)
        dense[g.gid] = v
    ms = oracle.Microstructure(shape, grains)
    cand = oracle.box_candidates(ms)
    for g in grains:
        m, idm = oracle.neighbour_max(g.gid, grains, phip, shape, 7.0)
        m2, idm2 = oracle.neighbour_max(g.gid, grains, phip, shape, 7.0, cand[g.gid])
        assert np.array_equal(m, m2) and np.array_equal(idm, idm2)
        pz, py, px = oracle.box_positions(g, shape)
        for (lz, z), (ly, y), (lx, x) in itertools.product(enumerate(pz), enumerate(py), enumerate(px)):
            others = [(dense[j, z, y, x], j) for j in range(len(grains)) if j != g.gid]
            best = max(v for v, _ in others)
            assert m[lz, ly, lx] == best
            ids = [j for v, j in others if v == best and v > -7.0]
            assert idm[lz, ly, lx] == (min(ids) if ids else -1)


def test_neighbour_max_tie_goes_to_lowest_id(oracle):
    shape = (1, 4, 4)
    a = oracle.Grain(0, (0, 0, 0), np.full((1, 4, 4), 1.0))
    b = oracle.Grain(1, (0, 0, 0), np.full((1, 4, 4), 2.0))
    c = oracle.Grain(2, (0, 0, 0), np.full((1, 4, 4), 2.0))
    grains = [a, b, c]
    phip = {g.gid: g.phi for g in grains}
    m, idm = oracle.neighbour_max(0, grains, phip, shape, 7.0)
    assert np.all(m == 2.0) and np.all(idm == 1)
    m, idm = oracle.neighbour_max(1, grains, phip, shape, 7.0)
    assert np.all(m == 2.0) and np.all(idm == 2)


def test_comparison_keeps_an_exact_sdf_pair(oracle):
    """Eq. (16): for two grains with phi_p_1 = d and phi_p_2 = -d the
    comparison returns d (and -d): the factor 1/2 keeps a signed distance a
    signed distance, and the pair stays antisymmetric."""
    rng = np.random.default_rng(5)
    d = rng.uniform(-6, 6, size=(3, 4, 5))
    assert np.allclose(oracle.compare(d, -d), d, atol=0)
    p1, p2 = rng.uniform(-7, 7, size=(2, 3, 4, 5))
    assert np.array_equal(oracle.compare(p1, p2), -oracle.compare(p2, p1))


# ---------------------------------------------------------- redistancing

def test_reference_value_is_exact_for_planes(oracle):
    """Sec. 2.1.6: reference cells get the exact distance to a planar
    interface when the plane crosses every axis within one cell."""
    rng = np.random.default_rng(6)
    for _ in range(5):
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        off = rng.uniform(8, 9)
        z, y, x = np.meshgrid(*(np.arange(16, dtype=float),) * 3, indexing="ij")
        d = nrm[2] * x + nrm[1] * y + nrm[0] * z - off - 0.0
        d = d + (8.0 - (nrm[2] * 8 + nrm[1] * 8 + nrm[0] * 8))   # plane through the middle
        ref, dref = oracle.reference_values(d, (False,) * 3, 7.0, (0, 1, 2))
        a = np.abs(d)
        every_axis = a < np.min(np.abs(nrm))
        interior = np.zeros(d.shape, bool)
        interior[1:-1, 1:-1, 1:-1] = True          # box faces see -eps outside (R5)
        sel = ref & every_axis & interior
        assert sel.sum() > 10
        assert np.max(np.abs(dref[sel] - a[sel])) < 1e-12


def _dijkstra_redistance(oracle, phic, full, eps, axes):
    """Multi-source shortest paths (scipy) over same-sign face neighbours with
    unit edges, sources = reference cells at their reference values."""
    pos = phic > 0
    ref, dref = oracle.reference_values(phic, full, eps, axes)
    shape = phic.shape
    n = phic.size
    idx = np.arange(n).reshape(shape)
    rows, cols, w = [], [], []
    for ax in axes:
        for k in (1,):
            nb = np.roll(idx, -k, axis=ax)
            ok = np.ones(shape, bool)
            if not full[ax]:
                sl = [slice(None)] * 3
                sl[ax] = slice(-k, None)
                ok[tuple(sl)] = False
            same = ok & (pos == np.roll(pos, -k, axis=ax))
            rows += list(idx[same]) + list(nb[same])
            cols += list(nb[same]) + list(idx[same])
            w += [1.0] * (2 * int(same.sum()))
    src = n
    for c in idx[ref]:
        rows.append(src)
        cols.append(int(c))
        w.append(1.0 + float(dref.flat[c]))    # offset by 1 so no weight is 0
    g = coo_matrix((w, (rows, cols)), shape=(n + 1, n + 1)).tocsr()
    dist = dijkstra(g, directed=True, indices=src)[:n] - 1.0
    mag = np.minimum(eps, dist).reshape(shape)
    mag = np.where(ref, dref, mag)
    return np.where(pos, mag, -mag)


@pytest.mark.parametrize("shape,full", [((6, 7, 5), (False,) * 3), ((5, 6, 7), (True, False, True)),
                                         ((1, 9, 8), (True, False, False))])
def test_redistance_fixed_point_is_shortest_path(oracle, shape, full):
    rng = np.random.default_rng(7)
    axes = oracle.spatial_axes(shape)
    for trial in range(4):
        phic = rng.uniform(-2, 2, size=shape) + rng.uniform(-1, 1)
        phic[rng.uniform(size=shape) < 0.05] = 0.0       # sign(0) = -1
        got = oracle.redistance(phic, full, 7.0, axes)
        ref = _dijkstra_redistance(oracle, phic, full, 7.0, axes)
        assert np.max(np.abs(got - ref)) < 1e-12
        assert np.array_equal(got > 0, phic > 0)


@pytest.mark.parametrize("shape,full", [((5, 6, 7), (False,) * 3), ((4, 6, 5), (True, True, False)),
                                         ((1, 11, 9), (False, False, True))])
def test_same_sign_restriction_is_immaterial(oracle, shape, full):
    """Every sign change lies between two reference cells, whose values are at
    most 1, so the same-sign fixed point equals the unrestricted taxicab
    distance transform of the classified magnitudes: min over all cells k of
    m_k + |x - k|_1 (minimum image on periodic axes), capped at eps, with the
    cell's own sign.  The pass kernels compute that transform with separable
    scans that ignore signs."""
    rng = np.random.default_rng(17)
    axes = oracle.spatial_axes(shape)
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"), -1).reshape(-1, 3)
    for trial in range(4):
        phic = rng.uniform(-3, 3, size=shape) + rng.uniform(-1, 1)
        phic[rng.uniform(size=shape) < 0.05] = 0.0
        is_ref, dref = oracle.reference_values(phic, full, 7.0, axes)
        m = np.where(is_ref, dref, 7.0).reshape(-1)
        d = np.abs(idx[:, None, :] - idx[None, :, :])
        for a in range(3):
            if full[a]:
                d[..., a] = np.minimum(d[..., a], shape[a] - d[..., a])
        brute = np.minimum(7.0, (m[None, :] + d.sum(-1)).min(axis=1)).reshape(shape)
        want = np.where(phic > 0, brute, -brute)
        got = oracle.redistance(phic, full, 7.0, axes)
        assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("shape,full", [((6, 13, 17), (False,) * 3), ((5, 16, 9), (True, True, False)),
                                         ((1, 21, 14), (False, False, True))])
def test_separable_windows_equal_the_transform(oracle, shape, full):
    """The kernels' form of that transform: one line at a time (x, then y,
    then z), each cell taking min over |k| <= 6 of m(x + k) + |k| (past the
    end of a non-periodic line eps, on a periodic one the wrapped cell).  As
    no magnitude exceeds eps = 7, a window of 6 steps is the whole line, and
    the three windowed passes give the unrestricted transform exactly."""
    rng = np.random.default_rng(23)
    axes = oracle.spatial_axes(shape)
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"), -1).reshape(-1, 3)
    for trial in range(3):
        phic = rng.uniform(-3, 3, size=shape) + rng.uniform(-1, 1)
        is_ref, dref = oracle.reference_values(phic, full, 7.0, axes)
        m = np.where(is_ref, dref, 7.0)
        d = np.abs(idx[:, None, :] - idx[None, :, :])
        for a in range(3):
            if full[a]:
                d[..., a] = np.minimum(d[..., a], shape[a] - d[..., a])
        brute = np.minimum(7.0, (m.reshape(-1)[None, :] + d.sum(-1)).min(axis=1)).reshape(shape)
        f = m.copy()
        for a in (2, 1, 0):                                 # x, y, z (array axes z, y, x)
            n = shape[a]
            if n == 1:
                continue
            out = f.copy()
            for k in range(1, 7):
                for sgn in (1, -1):
                    if full[a]:
                        nb = np.roll(f, -sgn * k, axis=a)
                    else:
                        nb = np.full_like(f, 7.0)
                        src = [slice(None)] * 3
                        dst = [slice(None)] * 3
                        if sgn > 0:
                            src[a], dst[a] = slice(k, None), slice(0, n - k)
                        else:
                            src[a], dst[a] = slice(0, n - k), slice(k, None)
                        nb[tuple(dst)] = f[tuple(src)]
                    out = np.minimum(out, nb + k)
            f = out
        assert np.max(np.abs(np.minimum(f, 7.0) - brute)) < 1e-12


def test_godunov_update_solves_the_upwind_equation(oracle):
    """R11: the closed-form update is the smallest root of
    sum_k max(u - a_k, 0)^2 = 1, found here by bisection instead."""
    rng = np.random.default_rng(21)
    for ndim in (1, 2, 3):
        a = [rng.uniform(0.0, 3.0, 400) for _ in range(ndim)]
        a[0][:50] = np.inf if ndim > 1 else a[0][:50]          # an axis without a neighbour
        u = oracle.godunov_update(a)
        lo = np.min(np.stack(a), axis=0)
        hi = lo + 1.0
        f = lambda v: sum(np.maximum(v - ak, 0.0) ** 2 for ak in a) - 1.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            neg = f(mid) < 0
            lo = np.where(neg, mid, lo)
            hi = np.where(neg, hi, mid)
        assert np.max(np.abs(u - 0.5 * (lo + hi))) < 1e-12


def test_godunov_redistance_is_euclidean_on_a_sphere(oracle):
    """R11 vs R5 on a sphere of radius 12 (distorted values, same zero level):
    the Godunov fixed point is first-order Euclidean (max error 0.38 cells in
    the band |d| <= 5), the taxicab one overshoots along diagonals (2.9)."""
    N, c = 40, 19.6
    z, y, x = np.meshgrid(*[np.arange(N, dtype=float)] * 3, indexing="ij")
    d = 12.0 - np.sqrt((x - c - 0.3) ** 2 + (y - c + 0.2) ** 2 + (z - c) ** 2)
    phic = np.clip(6.0 * np.tanh(d / 3.0), -7, 7)
    g = oracle.redistance_godunov(phic, (False,) * 3, 7.0, (0, 1, 2))
    t = oracle.redistance(phic, (False,) * 3, 7.0, (0, 1, 2))
    band = np.abs(d) <= 5.0
    assert np.abs(g - d)[band].max() < 0.45 and np.abs(g - d)[band].mean() < 0.12
    assert np.abs(t - d)[band].max() > 2.0
    assert np.array_equal(g > 0, phic > 0)


@pytest.mark.parametrize("shape,full", [((6, 7, 5), (False,) * 3), ((5, 6, 7), (True, False, True))])
def test_godunov_fixed_point(oracle, shape, full):
    """The returned magnitudes are a fixed point: reference cells keep their
    planar values, every other cell equals min(eps, update of its same-sign
    neighbours); an axis-aligned plane is reproduced exactly like R5."""
    rng = np.random.default_rng(22)
    axes = (0, 1, 2)
    phic = rng.uniform(-2, 2, size=shape) + rng.uniform(-1, 1)
    g = oracle.redistance_godunov(phic, full, 7.0, axes)
    is_ref, dref = oracle.reference_values(phic, full, 7.0, axes)
    mag, pos = np.abs(g), phic > 0
    mins = []
    for ax in axes:
        m = np.full(shape, np.inf)
        for k in (1, -1):
            nb = oracle._shift(mag, ax, k, full[ax], np.inf)
            ok = oracle._shift(np.ones(shape, bool), ax, k, full[ax], False) & (oracle._shift(pos, ax, k, full[ax], False) == pos)
            m = np.where(ok, np.minimum(m, nb), m)
        mins.append(m)
    want = np.where(is_ref, dref, np.minimum(7.0, oracle.godunov_update(mins)))
    assert np.max(np.abs(mag - want)) < 1e-12
    x = np.arange(30, dtype=float)
    d = np.broadcast_to(x - 12.3, (4, 5, 30)).copy()
    assert np.array_equal(oracle.redistance_godunov(np.clip(1.7 * d, -7, 7), (True, True, False), 7.0, axes),
                          oracle.redistance(np.clip(1.7 * d, -7, 7), (True, True, False), 7.0, axes))


def test_redistance_axis_plane_is_exact(oracle):
    """Taxicab propagation reproduces an axis-aligned planar SDF exactly
    (within eps) and caps it at eps."""
    x = np.arange(30, dtype=float)
    d = np.broadcast_to(x - 12.3, (4, 5, 30)).copy()
    d2 = np.clip(d * 1.7 + 0.05 * np.sin(x), -7, 7)      # same zero level, distorted values
    got = oracle.redistance(d2, (True, True, False), 7.0, (0, 1, 2))
    want = np.clip(d, -7, 7)
    # x in 6..19: one reference cell per side, then exact unit steps
    mid = slice(6, 20)
    assert np.max(np.abs(got[..., mid] - want[..., mid])) < 0.02
    assert np.array_equal(got > 0, d > 0)
    assert np.allclose(got[..., :4], -7.0)          # capped at -eps


# ---------------------------------------------------------------- box update

def test_box_update_is_bbox_plus_halo(oracle):
    shape = (20, 22, 24)
    rng = np.random.default_rng(8)
    for t in range(6):
        g = oracle.Grain(0, tuple(int(v) for v in rng.integers(0, 20, 3)),
                         np.full(tuple(int(v) for v in rng.integers(6, 15, 3)), -7.0))
        k = tuple(int(rng.integers(0, n)) for n in g.dims)
        g.phi[k] = 2.0
        g.phi[tuple(max(0, v - 1) for v in k)] = 1.0
        new = oracle.box_update(g, shape, 3, 7.0)
        # brute force: global cells of the positive set, bbox on the ring
        pz, py, px = oracle.box_positions(g, shape)
        cells = [(pz[a], py[b], px[c]) for a, b, c in zip(*np.nonzero(g.phi > 0))]
        for ax in range(3):
            n = shape[ax]
            loc = sorted(((c[ax] - g.origin[ax]) % n) for c in cells)
            ext = loc[-1] - loc[0] + 1 + 6
            if ext >= n:
                assert new.dims[ax] == n
            else:
                assert new.dims[ax] == ext
                assert new.origin[ax] == (g.origin[ax] + loc[0] - 3) % n
        # values travel with their global cell; other cells are -eps
        allpos = tuple(np.arange(s) for s in shape)
        vo, mo = oracle.sample(g, allpos, shape, -7.0)
        vn, mn = oracle.sample(new, allpos, shape, -7.0)
        assert np.array_equal(vn[mn], vo[mn])


def test_extinct_grain(oracle):
    g = oracle.Grain(3, (1, 2, 3), np.full((4, 4, 4), -1.0))
    assert not oracle.box_update(g, (10, 10, 10), 5, 7.0).alive


# ---------------------------------------------------------------- full steps

@pytest.mark.parametrize("halo", [7, 5])
def test_flat_bicrystal_is_stationary(oracle, halo):
    """P4: two grains split by two axis-aligned planes (periodic) do not move
    when the box offset covers the kernel radius plus one cell (the paper's
    7 cells, Fig. 1).  With a 5-cell halo the negative reference cell's
    convolution reads one cell of -eps beyond the box; the interface then
    drifts by less than 5e-4 cells per step."""
    n = 40
    shape = (8, 8, n)
    x = np.arange(n, dtype=float)
    d = np.minimum(x - 10.5, 29.5 - x)              # grain 0 between x=10.5 and 29.5
    d = np.broadcast_to(d, shape).copy()
    g0 = oracle.box_update(oracle.Grain(0, (0, 0, 0), np.clip(d, -7, 7)), shape, halo, 7.0)
    g1 = oracle.Grain(1, (0, 0, 0), np.clip(-d, -7, 7))
    ms = oracle.Microstructure(shape, [g0, g1], halo=halo)
    v0 = oracle.volumes(ms)
    ms2 = oracle.run(ms, 5, 1.0)
    area = 2 * 8 * 8
    if halo == 7:
        assert np.allclose(oracle.volumes(ms2), v0, rtol=0, atol=1e-9)
        for a, b in zip(ms.grains, ms2.grains):
            assert a.origin == b.origin and a.dims == b.dims
            assert np.max(np.abs(a.phi - b.phi)) < 1e-9
    else:
        drift = np.abs(oracle.volumes(ms2) - v0) / area / 5
        assert np.all(drift < 5e-4) and np.all(drift > 0)
        assert abs(oracle.volumes(ms2).sum() - v0.sum()) < 1e-6


def _sphere_slope(oracle, dim, n, r0, r_min, redist="taxicab"):
    shape = (n, n, n) if dim == 3 else (1, n, n)
    c = n / 2.0
    if dim == 3:
        fn = lambda z, y, x: r0 - np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    else:
        fn = lambda z, y, x: r0 - np.sqrt((x - c) ** 2 + (y - c) ** 2)
    ms = oracle.single_grain_state(shape, fn)
    ms.redist = redist
    ts, rs = [], []
    while True:
        v = oracle.volumes(ms)[0]
        r = (3 * v / (4 * math.pi)) ** (1 / 3) if dim == 3 else math.sqrt(v / math.pi)
        ts.append(ms.time)
        rs.append(r)
        if r < r_min or not ms.grains[0].alive:
            break
        ms = oracle.step(ms, 1.0)
    ts, rs = np.array(ts), np.array(rs)
    return np.polyfit(ts[rs >= r_min], rs[rs >= r_min] ** 2, 1)[0]


@pytest.mark.parametrize("dim,n,r0", [(2, 64, 20.0), (3, 40, 12.0)])
def test_sphere_law(oracle, dim, n, r0):
    """P1: r^2 = r0^2 - 2 (D-1) M gamma t.  With the paper's first-order
    (taxicab) redistancing the shrink rate is 20-24 % above the law at
    dt = 1 (the convolution samples the distorted band, Sec. 6.1); the test
    asserts the rate to lie in [1.0, 1.3] times the law, which a wrong kernel
    time, a wrong dimension factor or a sign error all leave."""
    slope = _sphere_slope(oracle, dim, n, r0, 5.0)
    law = -2.0 * (dim - 1)
    assert 1.0 <= slope / law <= 1.3, slope


@pytest.mark.parametrize("scheme", ["godunov", "hartmann"])
@pytest.mark.parametrize("dim,n,r0", [(2, 64, 20.0), (3, 40, 12.0)])
def test_sphere_law_other_reinitialisations(oracle, dim, n, r0, scheme):
    """P1 with the Godunov (R11) and the Hartmann (R16) re-initialisation: the
    Euclidean first-order propagation and the constrained reinitialization
    shrink the sphere at the taxicab scheme's rate to within 4 % (measured:
    1.23 and 1.21 vs 1.20 of the law in 2D, 1.21 and 1.19 vs 1.21 in 3D), so
    the excess over the law does not come from the taxicab metric or from the
    first-order band; the rate lies in [1.1, 1.3] times the law."""
    other = _sphere_slope(oracle, dim, n, r0, 5.0, scheme)
    taxi = _sphere_slope(oracle, dim, n, r0, 5.0)
    law = -2.0 * (dim - 1)
    assert 1.1 <= other / law <= 1.3, other
    assert abs(other / taxi - 1.0) <= 0.04, (other, taxi)


def test_von_neumann_mullins_2d(oracle):
    """P3: dA/dt = (pi/3) M gamma (n - 6) for 2D grains with n sides
    (Mullins 1956, cited in Sec. 4.1): fitted over jittered hexagonal grains,
    within the same 1.0-1.35 band as the sphere law."""
    N = 128
    seeds = I.jittered_hex_seeds(7, N, N, 8, 8, jitter=0.3)
    ms = oracle.tessellate((1, N, N), seeds)
    for _ in range(4):
        ms = oracle.step(ms, 1.0)

    def sides(ms):
        own = oracle.owner_map(ms)[0]
        nb = [set() for _ in ms.grains]
        for ax in (0, 1):
            o2 = np.roll(own, -1, axis=ax)
            m = own != o2
            for a, b in set(zip(own[m].tolist(), o2[m].tolist())):
                nb[a].add(b)
                nb[b].add(a)
        return np.array([len(s) for s in nb])
    n0 = sides(ms)
    a0 = oracle.volumes(ms)
    steps = 16
    ms = oracle.run(ms, steps, 1.0)
    n1 = sides(ms)
    keep = (n0 == n1) & np.array([g.alive for g in ms.grains])
    rate = (oracle.volumes(ms) - a0) / steps
    slope, icpt = np.polyfit(n0[keep] - 6, rate[keep], 1)
    assert 1.0 <= slope / (math.pi / 3) <= 1.35, slope
    assert abs(icpt) < 0.2


def test_magnetic_sphere_follows_ode(oracle):
    """P2: with a bulk energy difference dE the sphere obeys
    dr/dt = M (dE - 2 gamma / r) (3D, Eqs. (10), (19)): the bulk term adds
    M dE per unit time to the radial speed whatever the radius (checked as the
    difference of rates with and without dE), and a grain below the critical
    radius shrinks while one above it grows."""
    n = 44
    c = n / 2.0
    shape = (n, n, n)
    de = 0.25   # grain 0 has the lower energy: it is pushed outward

    def rate(r0, e):
        fn = lambda z, y, x: r0 - np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
        ms = oracle.single_grain_state(shape, fn)
        for g in ms.grains:
            g.idf = np.full(g.dims, 1 - g.gid, dtype=np.int64)
        ms.physics = oracle.isotropic_physics([0.0, e])
        v0 = oracle.volumes(ms)[0]
        ms = oracle.run(ms, 6, 1.0)
        v1 = oracle.volumes(ms)[0]
        return ((3 * v1 / (4 * math.pi)) ** (1 / 3) - (3 * v0 / (4 * math.pi)) ** (1 / 3)) / 6

    for r0 in (10.0, 14.0):
        bulk = rate(r0, de) - rate(r0, 0.0)
        assert 0.85 * de < bulk < 1.1 * de, (r0, bulk)
    assert rate(7.0, de) < 0 < rate(14.0, de)


def test_weighted_pair_moves_slower(oracle):
    """Eq. (10): a pair weight w scales the curvature motion by w."""
    n = 48
    c = n / 2.0
    fn = lambda z, y, x: 14.0 - np.sqrt((x - c) ** 2 + (y - c) ** 2)
    shape = (1, n, n)
    rates = {}
    for w in (1.0, 0.5):
        ms = oracle.single_grain_state(shape, fn)
        for g in ms.grains:
            g.idf = np.full(g.dims, 1 - g.gid, dtype=np.int64)
        ms.physics = oracle.Physics(weight=lambda i, j, w=w: (w, 1.0), energy=np.zeros(2))
        a0 = oracle.volumes(ms)[0]
        ms = oracle.run(ms, 10, 1.0)
        rates[w] = (oracle.volumes(ms)[0] - a0) / 10
    assert abs(rates[0.5] / rates[1.0] - 0.5) < 0.06


def test_volume_invariants_after_steps(oracle):
    """P5: after every step each cell has exactly one positive function, the
    voxel counts sum to N^D, and the smooth volumes sum to N^D within 0.5 %."""
    N = 32
    seeds = I.voronoi_seeds(5, 10, (N, N, N))
    ms = oracle.tessellate((N, N, N), seeds)
    for _ in range(3):
        ms = oracle.step(ms, 1.0)
        allpos = tuple(np.arange(N) for _ in range(3))
        npos = np.zeros((N, N, N), dtype=int)
        for g in ms.grains:
            if g.alive:
                v, _ = oracle.sample(g, allpos, ms.shape, -7.0)
                npos += v > 0
        assert np.all(npos == 1)
        assert oracle.voxel_counts(ms).sum() == N ** 3
        assert abs(oracle.volumes(ms).sum() - N ** 3) / N ** 3 < 5e-3


# ---------------------------------------------------------------- init

def test_labels_match_periodic_kdtree(oracle):
    N = 24
    seeds = I.voronoi_seeds(9, 30, (N, N, N))
    lab = oracle.labels_of_tessellation((N, N, N), seeds)
    tree = cKDTree(seeds, boxsize=[N, N, N])
    z, y, x = np.meshgrid(*(np.arange(N),) * 3, indexing="ij")
    pts = np.stack([x, y, z], -1).reshape(-1, 3).astype(float)
    _, idx = tree.query(pts)
    assert np.array_equal(lab.ravel(), idx)


def test_initial_sdf_two_seeds_is_plane_distance(oracle):
    """Reading R7 with two seeds: the initial function is the exact signed
    distance to the nearest bisector plane, positive on the grain's side."""
    N = 40
    seeds = np.array([[10.3, 20.0, 20.0], [29.7, 20.0, 20.0]])
    ms = oracle.tessellate((N, N, N), seeds)
    g = ms.grains[0]
    pz, py, px = oracle.box_positions(g, ms.shape)
    x = px.astype(float)
    # bisectors at x = 20 and x = 0 (= 40): distance to the nearer one
    want = np.minimum(20.0 - x, x - 0.0)
    want = np.where(x > 30, x - 40.0, want)
    got = g.phi[len(pz) // 2, len(py) // 2, :]
    assert np.allclose(got, np.clip(want, -7, 7), atol=1e-12)


def test_laguerre_weights_shift_the_bisector(oracle):
    """Power bisector: with weights w_i, w_j the plane moves by
    (w_i - w_j) / (2 |s_j - s_i|) toward grain j."""
    N = 40
    seeds = np.array([[10.0, 20.0, 20.0], [30.0, 20.0, 20.0]])
    w = np.array([40.0, 0.0])
    ms = oracle.tessellate((N, N, N), seeds, weights=w)
    g = ms.grains[0]
    pz, py, px = oracle.box_positions(g, ms.shape)
    got = g.phi[len(pz) // 2, len(py) // 2, :]
    x = px.astype(float)
    j = int(np.argmin(np.abs(x - 21.0)))
    assert abs(got[j] - (21.0 - x[j])) < 1e-12     # plane at x = 20 + 40/40 = 21


# ---------------------------------------------------------------- physics

def test_disorientation_cubic(oracle):
    def rot(axis, ang):
        axis = np.asarray(axis, float) / np.linalg.norm(axis)
        return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])
    e = np.array([1.0, 0, 0, 0])
    assert oracle.disorientation_cubic(e, e) < 1e-7
    assert abs(math.degrees(oracle.disorientation_cubic(e, rot([0, 0, 1], math.radians(30)))) - 30) < 1e-9
    assert abs(math.degrees(oracle.disorientation_cubic(e, rot([0, 0, 1], math.radians(60)))) - 30) < 1e-9
    assert oracle.disorientation_cubic(e, rot([1, 1, 1], math.radians(120))) < 1e-7
    q = I.random_quaternions(1, 200)
    angs = [math.degrees(oracle.disorientation_cubic(q[i], q[i + 1])) for i in range(199)]
    assert max(angs) <= 62.8 + 1e-6          # Mackenzie's maximum for cubic symmetry
    for s in oracle.cubic_symmetry_quaternions():
        a = oracle.disorientation_cubic(q[0], q[1])
        b = oracle.disorientation_cubic(q[0], oracle._qmul(q[1], s))
        assert abs(a - b) < 1e-9


def test_read_shockley_shape(oracle):
    tm = math.radians(15)
    assert oracle.read_shockley(tm, tm) == 1.0
    assert abs(oracle.read_shockley(tm / math.e, tm) - 2.0 / math.e) < 1e-15
    h = 1e-6
    slope = (oracle.read_shockley(tm * (1 - h), tm) - oracle.read_shockley(tm * (1 - 2 * h), tm)) / (h * tm)
    assert abs(slope) < 1e-4          # energy maximum at theta_max: smooth join to 1


def test_mobility_eq20_has_the_described_shape(oracle):
    """Sec. 4.1's prose around Eq. (20): low- and high-angle boundaries are
    distinguished, high angle above 15 degrees, with a steep ascent starting at
    8 degrees (reading R13: the printed formula completes its rise by 15
    degrees, not 10).  So: values in (0, 1], non-decreasing, a low-angle
    plateau up to 8 degrees (below 3 % of the high-angle mobility), the
    high-angle value (within 1 %) from 15 degrees on, and the half-way point
    of the rise between 8 and 15 degrees."""
    deg = math.radians(1.0)
    th = np.linspace(0.0, 62.8, 2000) * deg
    mu = np.array([oracle.mobility_eq20(t) for t in th])
    assert np.all(mu > 0.0) and np.all(mu <= 1.0)
    assert np.all(np.diff(mu) >= 0.0)
    assert np.all(mu[th <= 8 * deg] < 0.03)
    assert np.all(mu[th >= 15 * deg] > 0.99)
    half = th[np.argmax(mu >= 0.5)]
    assert 8 * deg < half < 15 * deg


def test_magnetic_energy_matches_printed_maximum(oracle):
    """P7: Eq. (18) with the printed B = 17 T and dchi = 1.18e-5 gives the
    largest orientation energy; the paper's printed maximum 1351.23 J/m^3
    (its most field-parallel grain) lies 0.42 % below the cos^2 = 1 value."""
    gc = json.load(open(GOLDEN))["magnetic_ti"]
    e1 = oracle.magnetic_energy_density(gc["B_tesla"], gc["dchi"], 1.0)
    assert abs(e1 - 1356.88) < 0.01
    assert 0 < (e1 - gc["E_m_max_printed"]) / e1 < 0.005
    assert oracle.magnetic_energy_density(gc["B_tesla"], gc["dchi"], 0.0) == 0.0


def test_c_axis_rotation(oracle):
    q = np.array([math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0, 0.0])   # 90 deg about x
    assert np.allclose(oracle.c_axis(q), [0, -1, 0], atol=1e-15)


# ---------------------------------------------------------------- inputs

def test_splitmix64_reference_values():
    """SplitMix64 from seed 0: published first outputs of the generator."""
    got = [int(v) for v in I.u64(0, np.arange(3))]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# ---------------------------------------------------------------- grain statistics

def test_grain_statistics_closed_forms(oracle):
    """Equal spheres: <R> = R, rms = R, all in the bin of R / <R> = 1; two
    sizes in 2D: the equivalent radii of the disc areas and their mean; extinct
    (V = 0) grains are not counted; ratios at or above r_max overflow."""
    r0 = 4.0
    v = np.array([4.0 / 3.0 * math.pi * r0 ** 3] * 5 + [0.0, 0.0])
    st = oracle.grain_statistics(v, 3, 10, 2.0)
    assert st["alive"] == 5
    assert abs(st["mean_radius"] - r0) < 1e-12 and abs(st["rms_radius"] - r0) < 1e-12
    assert st["hist"][5] == 1.0 and st["hist"].sum() == 1.0 and st["overflow"] == 0.0
    a = np.array([math.pi * 1.0, math.pi * 9.0, 0.0])             # discs of radius 1 and 3
    st = oracle.grain_statistics(a, 2, 4, 1.4)
    assert st["alive"] == 2 and abs(st["mean_radius"] - 2.0) < 1e-12
    assert abs(st["rms_radius"] - math.sqrt(5.0)) < 1e-12 and st["max_radius"] == 3.0
    assert st["hist"][1] == 0.5 and st["overflow"] == 0.5         # 0.5 in [0.35, 0.7); 1.5 >= 1.4
    assert abs(st["mean_volume"] - 5.0 * math.pi) < 1e-12



# ---------------------------------------------------------------- grid coarsening (Sec. 4.1, R12)

def _box_grain(oracle, shape, origin, dims, seed, eps=7.0):
    rng = np.random.default_rng(seed)
    return oracle.Grain(0, tuple(origin), rng.uniform(-eps, eps, size=tuple(dims)))


def test_coarse_project_identity_ratio_pads_with_fill(oracle):
    """N' = N: u = i', every weight is 0, so the projection is the box's own
    values, and the coarse box adds one cell of -eps on each side."""
    shape = (20, 22, 24)
    g = _box_grain(oracle, shape, (3, 4, 5), (9, 8, 7), 1)
    p = oracle.coarse_project(g, shape, shape, 7.0)
    assert p.origin == (2, 3, 4)
    want = np.pad(g.phi, 1, constant_values=-7.0)
    assert p.phi.shape == want.shape
    assert np.array_equal(p.phi, want)


def test_coarse_project_half_ratio_takes_even_cells(oracle):
    """N' = N / 2 on a full-domain box: coarse cell i' sits on fine cell 2 i'
    exactly, so the projection is half the fine value there."""
    shape = (16, 20, 24)
    g = _box_grain(oracle, shape, (0, 0, 0), shape, 2)
    p = oracle.coarse_project(g, shape, (8, 10, 12), 7.0)
    assert p.origin == (0, 0, 0)
    assert np.array_equal(p.phi, 0.5 * g.phi[::2, ::2, ::2])


def test_coarse_project_reproduces_affine_functions(oracle):
    """Trilinear interpolation is exact on affine functions: with N' / N = 2/3
    (u = 1.5 i'), a box holding a z + b y + c x + d (distinct slopes per axis,
    so a swapped axis shows) projects to (2/3)(a u_z + b u_y + c u_x + d)
    wherever all eight corners lie in the box."""
    shape, shape2, eps = (48, 48, 48), (32, 32, 32), 1e6
    o, n = (6, 9, 12), (30, 27, 24)
    a, b, c, d = 0.37, -0.21, 0.113, 1.5
    z, y, x = np.meshgrid(*[o[k] + np.arange(n[k]) for k in range(3)], indexing="ij")
    g = oracle.Grain(0, o, a * z + b * y + c * x + d)
    p = oracle.coarse_project(g, shape, shape2, eps)
    uz, uy, ux = np.meshgrid(*[(p.origin[k] + np.arange(p.phi.shape[k])) * 1.5 for k in range(3)], indexing="ij")
    inside = np.ones(p.phi.shape, dtype=bool)
    for u, k in ((uz, 0), (uy, 1), (ux, 2)):
        inside &= (np.floor(u) >= o[k]) & (np.floor(u) + 1 <= o[k] + n[k] - 1)
    assert inside.sum() > 1000
    want = (2.0 / 3.0) * (a * uz + b * uy + c * ux + d)
    assert np.max(np.abs(p.phi[inside] - want[inside])) < 1e-12


def test_coarse_project_matches_scipy_linear_interpolation(oracle):
    """The projection equals scipy's periodic linear interpolation
    (map_coordinates, order 1, grid-wrap) of the fine field (-eps outside the
    box) at u = i' N / N', times N' / N; and every coarse cell that the box
    influences lies in the coarse box, which includes boxes crossing the
    periodic boundary."""
    ndimage = pytest.importorskip("scipy.ndimage")
    shape, shape2, eps = (30, 36, 42), (20, 24, 28), 7.0
    for seed, origin, dims in ((3, (25, 2, 30), (11, 13, 17)), (4, (0, 20, 5), (9, 16, 20))):
        g = _box_grain(oracle, shape, origin, dims, seed)
        fine = np.full(shape, -eps)
        idx = np.ix_(*[(origin[k] + np.arange(dims[k])) % shape[k] for k in range(3)])
        fine[idx] = g.phi
        coords = np.meshgrid(*[np.arange(shape2[k]) * shape[k] / shape2[k] for k in range(3)], indexing="ij")
        full = (2.0 / 3.0) * ndimage.map_coordinates(fine, coords, order=1, mode="grid-wrap")
        p = oracle.coarse_project(g, shape, shape2, eps)
        pidx = np.ix_(*[(p.origin[k] + np.arange(p.phi.shape[k])) % shape2[k] for k in range(3)])
        assert np.max(np.abs(p.phi - np.clip(full[pidx], -eps, eps))) < 1e-12
        outside = np.ones(shape2, dtype=bool)
        outside[pidx] = False
        assert np.all(np.abs(full[outside] + (2.0 / 3.0) * eps) < 1e-12)


def test_coarsen_halves_a_sphere_exactly(oracle):
    """A sphere of radius 10 about fine cell (24, 24, 24), coarsened 48 -> 24:
    coarse cells sit on even fine cells, so the coarse grain's positive set is
    exactly the lattice sphere of radius 5 about (12, 12, 12); near the
    surface the re-initialised values are the planar-exact distances (within
    0.1 of the Euclidean ones), further out taxicab distances (between the
    Euclidean distance and sqrt(3) times it); the box is the bbox of the
    positive set (|i' - 12| <= 4) plus the halo of 5."""
    shape = (48, 48, 48)
    ms = oracle.single_grain_state(
        shape, lambda z, y, x: 10.0 - np.sqrt((z - 24) ** 2 + (y - 24) ** 2 + (x - 24) ** 2))
    c = oracle.coarsen(ms, (24, 24, 24))
    g = c.grains[0]
    z, y, x = np.meshgrid(*[np.arange(24)] * 3, indexing="ij")
    r = np.sqrt((z - 12.0) ** 2 + (y - 12.0) ** 2 + (x - 12.0) ** 2)
    val, _ = oracle.sample(g, (np.arange(24),) * 3, (24, 24, 24), -7.0)
    assert np.array_equal(val > 0, r < 5.0)
    shell = np.abs(r - 5.0) < 0.5
    assert np.max(np.abs(val[shell] - (5.0 - r[shell]))) < 0.1
    band = np.abs(r - 5.0) < 3.0
    e, t = np.abs(5.0 - r[band]), np.abs(val[band])
    assert np.all(t >= e - 0.1) and np.all(t <= math.sqrt(3.0) * e + 0.1)
    assert g.origin == (3, 3, 3) and g.dims == (19, 19, 19)
    assert c.grains[1].dims == (24, 24, 24)       # the complement grain keeps a full box


def test_coarsen_rebuilds_the_id_field(oracle):
    """With physics, coarsening rebuilds the ID-field (R3 / R4) from the coarse
    functions: in a sphere + complement pair, the sphere's ID-field is the
    complement (id 1) wherever the complement's coarse value exceeds -eps,
    -1 elsewhere; it is carried into the new box like phi (-1 in the cells the
    box update adds beyond the coarse box it was computed on)."""
    shape = (40, 40, 40)
    ms = oracle.single_grain_state(
        shape, lambda z, y, x: 8.0 - np.sqrt((z - 20) ** 2 + (y - 20) ** 2 + (x - 20) ** 2))
    ms.physics = oracle.isotropic_physics(np.zeros(2))
    c = oracle.coarsen(ms, (20, 20, 20))
    g0, g1 = c.grains
    assert g0.idf is not None and g0.idf.shape == g0.phi.shape
    pos = oracle.box_positions(g0, (20, 20, 20))
    other, _ = oracle.sample(g1, pos, (20, 20, 20), -7.0)
    cb = [oracle.coarse_axis(ms.grains[0].origin[a], ms.grains[0].dims[a], 40, 20) for a in range(3)]
    inside = np.ones(g0.dims, dtype=bool)
    for a in range(3):
        sh = [1, 1, 1]
        sh[a] = -1
        inside &= (((pos[a] - cb[a][0]) % 20) < cb[a][1]).reshape(sh)
    assert np.array_equal(g0.idf, np.where(inside & (other > -7.0), 1, -1))
    assert (g0.idf == 1).any() and (~inside).any()


# ---------------------------------------------------------------- size analysis (Sec. 5, R14)

def _quad(f, a, b):
    integrate = pytest.importorskip("scipy.integrate")
    return integrate.quad(f, a, b, limit=400)[0]


def test_rios_is_a_density_with_the_printed_moments(oracle):
    """Eq. (Rios) with H = 3 integrates to 1 for any 0 < nu < 4 (this fixes
    the garbled nu exponent, R14), and at the paper's steady state
    (nu = 3.106, rho = 0.863) has E(z) = 1 and Var(z) = 1/rho - 1
    (Eq. (varianz)) to the precision the paper's 'approximately' allows."""
    c = json.load(open(GOLDEN))["size_distribution"]
    for nu, rho in ((3.106, 0.863), (2.5, 0.8), (3.9, 0.85), (1.0, 0.7)):
        assert abs(_quad(lambda z: float(oracle.rios_pdf(z, nu, rho)), 0.0, np.inf) - 1.0) < 1e-8
    nu, rho = c["steady_nu"], c["steady_rho"]
    m1 = _quad(lambda z: z * float(oracle.rios_pdf(z, nu, rho)), 0.0, np.inf)
    m2 = _quad(lambda z: z * z * float(oracle.rios_pdf(z, nu, rho)), 0.0, np.inf)
    assert abs(m1 - 1.0) < 5e-3
    assert abs((m2 - m1 * m1) - (1.0 / rho - 1.0)) < 0.02 * (1.0 / rho - 1.0)


def test_rios_tends_to_hillert(oracle):
    """Sec. 5: nu -> 4 with rho = 8/9 gives Hillert's distribution; Hillert's
    density (written independently from its own closed form) integrates to
    1 with E(z) = 1 and Var(z) = 1/8 = 1/rho - 1."""
    rho = json.load(open(GOLDEN))["size_distribution"]["hillert_rho"]
    z = np.linspace(0.02, 2.4, 200)
    for d in (1e-3, 1e-5, 1e-7):
        err = np.max(np.abs(oracle.rios_pdf(z, 4.0 - d, rho) - oracle.hillert_pdf(z)))
        assert err < 30.0 * d, (d, err)
    top = 2.0 / rho
    assert abs(_quad(lambda q: float(oracle.hillert_pdf(q)), 0.0, top) - 1.0) < 1e-10
    assert abs(_quad(lambda q: q * float(oracle.hillert_pdf(q)), 0.0, top) - 1.0) < 1e-10
    var = _quad(lambda q: q * q * float(oracle.hillert_pdf(q)), 0.0, top) - 1.0
    assert abs(var - (1.0 / rho - 1.0)) < 1e-10


def test_grain_statistics_rho_and_variance(oracle):
    """Radii 1 and 3: <R> = 2, <R^2> = 5, so rho = 4/5 and Var(z) = 1/4 =
    1/rho - 1 exactly."""
    vol = np.array([4.0 / 3.0 * math.pi, 4.0 / 3.0 * math.pi * 27.0, 0.0])
    st = oracle.grain_statistics(vol, 3, 10, 3.0)
    assert abs(st["rho"] - 0.8) < 1e-14
    assert abs(st["var_z"] - 0.25) < 1e-14


def test_growth_exponent_fit_recovers_the_law(oracle):
    """Exact series of <R>^(1/n) - <R_0>^(1/n) = k t: the fit returns (n, k),
    for the parabolic law (n = 1/2) and for the paper's n = 0.458."""
    t = np.linspace(0.0, 400.0, 60)
    for n, k, r0 in ((0.5, 0.7, 3.0), (0.458, 0.21, 5.0)):
        r = (r0 ** (1.0 / n) + k * t) ** n
        fn, fk = oracle.fit_growth_exponent(t, r)
        assert abs(fn - n) < 1e-6 and abs(fk - k) < 1e-5 * k, (n, fn, k, fk)


def test_rios_nu_fit_recovers_nu(oracle):
    """A histogram of Eq. (Rios)'s bin-centre densities at the paper's
    steady state returns its nu."""
    c = json.load(open(GOLDEN))["size_distribution"]
    n_bins, r_max = 30, 3.0
    zc = (np.arange(n_bins) + 0.5) * (r_max / n_bins)
    hist = oracle.rios_pdf(zc, c["steady_nu"], c["steady_rho"]) * (r_max / n_bins)
    assert abs(oracle.fit_rios_nu(hist, r_max, c["steady_rho"]) - c["steady_nu"]) < 1e-5


def test_texture_shares_by_hand(oracle):
    vol = np.array([10.0, 30.0, 0.0, 60.0])
    cls = np.array([0, 1, 1, -1])
    assert np.allclose(oracle.texture_shares(vol, cls, 2), [0.1, 0.3], rtol=0, atol=1e-15)


# ------------------------------------------------- anisotropy map (R15)

def _tri_area(T):
    return 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1)


def test_gb_triangles_of_an_oblique_plane_are_exact(oracle):
    """A linear function's zero level is triangulated exactly: every vertex
    lies on the plane, and the area is the plane's section of the box
    (width (ny-1), length (nx-1)/cos theta for a plane tilted in z-x)."""
    nz, ny, nx = 12, 7, 9
    th = 0.35
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = 5.2 - (z * math.cos(th) + x * math.sin(th))       # crosses x = 0 .. nx-1 inside z's range
    T, g = oracle.gb_triangles(phi, np.where(phi <= 0, 3, -1))
    on = T[..., 0] * math.cos(th) + T[..., 2] * math.sin(th) - 5.2
    assert np.abs(on).max() < 1e-12
    assert abs(_tri_area(T).sum() - (ny - 1) * (nx - 1) / math.cos(th)) < 1e-9
    assert set(g.tolist()) == {3}


def _sphere(n, r, c):
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    return r - np.sqrt((z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2)


def test_gb_triangles_of_a_sphere_are_a_closed_sphere(oracle):
    """The triangulated zero level of a sphere's distance function is a closed
    2-manifold of Euler characteristic 2 (every edge in exactly two
    triangles), its vertices within the chord error of radius r, and its area
    within 1% of 4 pi r^2."""
    r, c = 8.3, (12.4, 11.7, 12.1)
    T, _ = oracle.gb_triangles(_sphere(26, r, c), np.zeros((26, 26, 26), dtype=np.int64))
    rad = np.linalg.norm(T - np.array(c), axis=2)
    assert np.abs(rad - r).max() < 3.0 / (8.0 * r) + 1e-9      # longest tetrahedron edge sqrt(3)
    assert abs(_tri_area(T).sum() / (4 * math.pi * r * r) - 1.0) < 0.01
    key = {}
    vid = np.array([key.setdefault(tuple(np.round(v, 9)), len(key)) for v in T.reshape(-1, 3)]).reshape(-1, 3)
    edges = {}
    for a, b, cc in vid:
        for e in ((a, b), (b, cc), (cc, a)):
            e = (min(e), max(e))
            edges[e] = edges.get(e, 0) + 1
    assert set(edges.values()) == {2}
    assert len(key) - len(edges) + len(vid) == 2


def test_point_triangle_distance_matches_brute_force(oracle):
    """Against the minimum over a fine barycentric sample of each triangle:
    never above it, and below it by at most the sample's spacing; collinear
    (degenerate) triangles included."""
    rng = np.random.default_rng(15)
    tris = rng.uniform(-2, 2, (40, 3, 3))
    tris[0, 2] = 0.5 * (tris[0, 0] + tris[0, 1])               # degenerate
    s = np.linspace(0.0, 1.0, 161)
    a, b = np.meshgrid(s, s, indexing="ij")
    keep = a + b <= 1.0
    bary = np.stack([1 - a[keep] - b[keep], a[keep], b[keep]], 1)
    for p in rng.uniform(-3, 3, (25, 3)):
        d = oracle.point_triangle_distance(p, tris)
        for k in range(len(tris)):
            pts = bary @ tris[k]
            dmin = np.linalg.norm(pts - p, axis=1).min()
            diam = max(np.linalg.norm(tris[k, i] - tris[k, j]) for i in range(3) for j in range(3))
            assert d[k] <= dmin + 1e-12 and d[k] >= dmin - diam / 160.0, (k, d[k], dmin)


def test_closest_gb_distance_is_the_sphere_distance(oracle):
    """Every band cell of a sphere grain lies at distance |r - |p - c|| from
    the true boundary; the closest triangle gives it within the chord error."""
    r, c = 7.6, (10.3, 9.8, 10.2)
    phi = _sphere(21, r, c)
    T, _ = oracle.gb_triangles(phi, np.zeros(phi.shape, dtype=np.int64))
    for z, y, x in zip(*np.nonzero(np.abs(phi) < 2.5)):
        d = oracle.point_triangle_distance(np.array([z, y, x], dtype=np.float64), T).min()
        assert abs(d - abs(phi[z, y, x])) < 3.0 / (8.0 * (r - 2.5)) + 0.02


def test_closest_gb_grains_at_a_triple_junction(oracle):
    """Grain 0 fills x < 9.5; across its plane boundary grain 1 holds y <= 7
    and grain 2 y >= 8 (the junction line at y = 7.5).  Every band cell adopts
    the grain straight across the plane: 1 for y <= 6, 2 for y >= 9, either at
    the junction.  A sentinel id on grain 0's own side must never be adopted
    (the label comes from the corners outside the grain)."""
    nz, ny, nx = 5, 16, 20
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = np.clip(9.5 - x, -7.0, 7.0).astype(np.float64)
    across = np.where(y <= 7, 1, 2)
    idf = np.where(phi <= 0, across, 5)
    out = oracle.closest_gb_grains(phi, idf, 3.0)
    band = np.abs(phi) < 3.0
    assert np.all(out[~band] == idf[~band])
    assert np.all(out[band & (y <= 6)] == 1) and np.all(out[band & (y >= 9)] == 2)
    assert set(np.unique(out[band & ((y == 7) | (y == 8))]).tolist()) <= {1, 2}


def test_closest_gb_grains_of_a_bicrystal_and_an_isolated_grain(oracle):
    """A bicrystal: every band cell adopts the one neighbour.  No boundary in
    the box (all positive) or no neighbour (-1 outside): the map is the
    ID-field, resp. -1 (w = 1)."""
    phi = np.clip(4.5 - np.arange(10), -7, 7)[None, None, :] * np.ones((3, 4, 1))
    idf = np.where(phi <= 0, 4, 4)
    out = oracle.closest_gb_grains(phi, idf, 2.0)
    assert np.all(out == 4)
    assert np.array_equal(oracle.closest_gb_grains(np.full((3, 3, 3), 2.0), np.full((3, 3, 3), 6), 3.0),
                          np.full((3, 3, 3), 6))
    out = oracle.closest_gb_grains(phi, np.full(phi.shape, -1), 2.0)
    assert np.all(out == -1)


# ------------------------------------------------- initial boxes and signs (R6, R7)

def _min_arc(coords, n):
    """Brute force: the shortest arc (start, length) of the n-cycle that covers
    every coordinate, the smallest start among the shortest."""
    occ = {int(c) % n for c in coords}
    for length in range(1, n + 1):
        for start in range(n):
            if occ <= {(start + k) % n for k in range(length)}:
                return start, length


@pytest.mark.parametrize("shape,n,seed", [((20, 24, 28), 18, 21), ((1, 40, 36), 25, 22)])
def test_initial_boxes_are_tight_periodic_bboxes(oracle, shape, n, seed):
    """Every grain's initial box is the shortest periodic arc of its label
    cells per axis, grown by the halo on both sides (the whole axis once that
    reaches N), found here by brute force over all arcs."""
    seeds = I.voronoi_seeds(seed, n, (shape[2], shape[1], shape[0]))
    ms = oracle.tessellate(shape, seeds, halo=3)
    lab = oracle.labels_of_tessellation(shape, seeds)
    for g in ms.grains:
        cells = np.argwhere(lab == g.gid)
        if len(cells) == 0:
            assert not g.alive
            continue
        for a in range(3):
            if shape[a] == 1:
                assert g.dims[a] == 1
                continue
            s, length = _min_arc(cells[:, a], shape[a])
            if length + 6 >= shape[a]:
                assert g.dims[a] == shape[a]
            else:
                assert g.dims[a] == length + 6 and g.origin[a] == (s - 3) % shape[a], (g.gid, a)


def test_initial_functions_agree_with_the_labels(oracle):
    """R7: a grain's initial function is >= 0 on its own label cells (<= its
    distance to every bisector plane of a face neighbour, all of which it is
    on the grain's side of) and <= 0 on the cells of its face neighbours."""
    shape = (18, 22, 20)
    seeds = I.voronoi_seeds(31, 20, (shape[2], shape[1], shape[0]))
    ms = oracle.tessellate(shape, seeds)
    lab = oracle.labels_of_tessellation(shape, seeds)
    nbs = oracle.face_neighbours(lab, len(seeds))
    checked = 0
    for g in ms.grains:
        if not g.alive:
            continue
        pz, py, px = oracle.box_positions(g, shape)
        L = lab[np.ix_(pz, py, px)]
        assert np.all(g.phi[L == g.gid] >= -1e-12)
        nb = np.isin(L, list(nbs[g.gid]))
        assert np.all(g.phi[nb] <= 1e-12)
        checked += int(nb.sum())
    assert checked > 1000


def test_gb_map_takes_the_pair_from_the_closest_boundary(oracle):
    """R15 in Eq. (10): a cylinder grain whose outside belongs to grain 1
    (x < c) and grain 2 (x >= c), with w(0, 1) = 1 and w(0, 2) = 0.5, and no
    ID entry on its own cells (-1: w = 1 under R3).  With the map each band
    cell blends with the weight of the grain across its closest boundary
    point: its change is exactly w(map) times the R3 change, 0.5 on the x > c
    side; isotropic physics is unaffected by the map."""
    shape, c = (4, 40, 40), 19.6
    ms = oracle.single_grain_state(shape, lambda z, y, x: 11.0 - np.sqrt((x - c) ** 2 + (y - 19.3) ** 2))
    g = ms.grains[0]
    pz, py, px = oracle.box_positions(g, shape)
    X = np.broadcast_to(px[None, None, :], g.dims)
    g.idf = np.where(g.phi <= 0, np.where(X < c, 1, 2), -1).astype(np.int64)
    taps = oracle.heat_kernel_taps(1.0, 5)
    wts = {1: 1.0, 2: 0.5}
    r3 = oracle.Physics(weight=lambda i, j: (wts[j], 1.0), energy=np.zeros(3))
    r15 = oracle.Physics(weight=lambda i, j: (wts[j], 1.0), energy=np.zeros(3), gb_map_tube=3.0)
    p3 = oracle.predict(g, shape, taps, ms.eps, r3, 1.0)
    p15 = oracle.predict(g, shape, taps, ms.eps, r15, 1.0)
    m = oracle.closest_gb_grains(g.phi, g.idf, 3.0)
    band = (np.abs(g.phi) < 3.0) & (g.phi > 0)
    assert np.all(m[band & (X > c + 1.5)] == 2) and np.all(m[band & (X < c - 1.5)] == 1)
    w = np.where(m == 2, 0.5, 1.0)
    assert np.allclose((p15 - g.phi)[band], (w * (p3 - g.phi))[band], rtol=0, atol=1e-12)
    assert np.abs((p15 - g.phi)[band & (X > c + 1.5)]).max() > 1e-3
    iso = lambda tube: oracle.Physics(weight=lambda i, j: (1.0, 1.0), energy=np.zeros(3), gb_map_tube=tube)
    assert np.array_equal(oracle.predict(g, shape, taps, ms.eps, iso(None), 1.0),
                          oracle.predict(g, shape, taps, ms.eps, iso(3.0), 1.0))


# ---------------------------------------------------------------- R16 (Hartmann)

def _hcr_sphere(n=28, c=13.7, r0=8.0):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((z - c) ** 2 + (y - c) ** 2 + (x - c) ** 2)
    return r0 - r, r


def _crossing_shift(p0, out):
    """Largest move of a linearly interpolated zero crossing between face
    neighbours of opposite sign in p0 (fraction of a cell)."""
    worst = 0.0
    for ax in range(3):
        a0, a1 = p0, np.roll(p0, -1, axis=ax)
        b0, b1 = out, np.roll(out, -1, axis=ax)
        m = (a0 > 0) != (a1 > 0)
        last = [slice(None)] * 3
        last[ax] = p0.shape[ax] - 1
        m[tuple(last)] = False
        worst = max(worst, float(np.max(np.abs(a0[m] / (a0[m] - a1[m]) - b0[m] / (b0[m] - b1[m])))))
    return worst


@pytest.mark.parametrize("kind", ["sdf", "same_zero_level", "scaled"])
def test_hartmann_reinitialisation_on_a_sphere(oracle, kind):
    """R16: from the exact signed distance of a sphere of radius 8, from a
    function with the same zero level but |grad phi| != 1 ((r0^2 - r^2) /
    2 r0) and from twice the distance, the constrained reinitialization gives
    the distance to within 0.1 cells next to the surface and 0.35 within 4
    cells (the taxicab scheme: about 0.46 and 2.6), keeps every cell's sign
    and moves no interpolated zero crossing by more than 0.08 of a cell.
    Each of a flipped S, an inverted constraint ratio, swapped upwind
    branches and a flipped or missing forcing term fails these bounds."""
    eps = 7.0
    sd, r = _hcr_sphere()
    p0 = {"sdf": sd, "same_zero_level": (64.0 - r * r) / 16.0, "scaled": 2.0 * sd}[kind]
    p0 = np.clip(p0, -eps, eps)
    out = oracle.redistance_hartmann(p0, (False,) * 3, eps, (0, 1, 2))
    near, band = np.abs(sd) <= 1.0, np.abs(sd) <= 4.0
    assert np.max(np.abs(out - sd)[near]) < 0.1
    assert np.max(np.abs(out - sd)[band]) < 0.35
    taxi = oracle.redistance(p0, (False,) * 3, eps, (0, 1, 2))
    assert np.max(np.abs(out - sd)[band]) < 0.5 * np.max(np.abs(taxi - sd)[band])
    assert np.array_equal(out > 0, p0 > 0)
    assert _crossing_shift(p0, out) < 0.08


@pytest.mark.parametrize("axis", [0, 2])
def test_hartmann_planar_slab_is_stationary(oracle, axis):
    """R16: a slab grain bounded by two planes normal to one axis, the box full
    and periodic along the other two, its function the clamped distance: the
    upwind |grad phi| is 1, every constraint ratio is already met, so the
    reinitialization leaves it unchanged."""
    eps, n = 7.0, 30
    coord = np.arange(n, dtype=np.float64) - 0.3
    d1 = np.minimum(coord - 9.0, 20.0 - coord)
    shape = [6, 6, 6]
    shape[axis] = n
    bshape = [1, 1, 1]
    bshape[axis] = n
    phi = np.broadcast_to(np.clip(d1, -eps, eps).reshape(bshape), shape).copy()
    full = tuple(a != axis for a in range(3))
    out = oracle.redistance_hartmann(phi, full, eps, (0, 1, 2))
    assert np.max(np.abs(out - phi)) < 1e-12


def test_godunov_gradient_norm_of_planes_and_a_kink(oracle):
    """The upwind |grad phi| of R16: 1 at every interior cell of a unit-slope
    oblique linear function on both sides of its zero level; at the kink of
    a ridge where S > 0 and of a valley where S < 0 (the cells farthest from
    the zero level, reached from both sides) 1 as well, and 0 at the bottom
    of a valley where S > 0 (no neighbour lies upwind of it)."""
    n = 10
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    nv = np.array([2.0, 3.0, 6.0]) / 7.0
    lin = nv[0] * (z - 4.2) + nv[1] * (y - 3.9) + nv[2] * (x - 5.1)
    g = oracle.godunov_gradient_norm(lin, lin, (False,) * 3, 7.0, (0, 1, 2))
    inner = (slice(1, -1),) * 3
    assert np.max(np.abs(g[inner] - 1.0)) < 1e-12
    v = np.abs(x - 4.5).astype(np.float64)
    pos, neg = np.ones_like(v), -np.ones_like(v)
    ridge = oracle.godunov_gradient_norm(6.0 - v, pos, (True, True, False), 7.0, (0, 1, 2))
    assert np.max(np.abs(ridge[:, :, 1:-1] - 1.0)) < 1e-12
    valley = oracle.godunov_gradient_norm(v - 6.0, neg, (True, True, False), 7.0, (0, 1, 2))
    assert np.max(np.abs(valley[:, :, 1:-1] - 1.0)) < 1e-12
    bottom = oracle.godunov_gradient_norm(v + 1.0, pos, (True, True, False), 7.0, (0, 1, 2))
    assert np.all(bottom[:, :, 4:6] == 0.0) and np.max(np.abs(bottom[:, :, 1:4] - 1.0)) < 1e-12


def test_hartmann_without_a_zero_level_keeps_the_clamp(oracle):
    """R16: a box with no positive cell has no constrained cell; its clamped
    -eps function stays as it is."""
    neg = np.full((8, 9, 10), -7.0)
    assert np.array_equal(oracle.redistance_hartmann(neg, (False,) * 3, 7.0, (0, 1, 2)), neg)


def test_point_triangle_distances_equal_the_single_point_form(oracle):
    """The block form of the point-triangle distance (used by the map over many
    cells) equals the single-point form row by row, bit for bit, on random
    points and triangles, degenerate ones included; and the map's blocked
    search equals a cell-by-cell search on a tessellation box."""
    rng = np.random.default_rng(3)
    tris = rng.uniform(-2, 2, (60, 3, 3))
    tris[5, 2] = tris[5, 1]                           # a segment
    tris[6, 1] = tris[6, 0]
    tris[6, 2] = tris[6, 0]                           # a point
    tris[7, 2] = tris[7, 0] + 2.0 * (tris[7, 1] - tris[7, 0])   # collinear
    pts = rng.uniform(-3, 3, (40, 3))
    block = oracle.point_triangle_distances(pts, tris)
    for k, p in enumerate(pts):
        assert np.array_equal(block[k], oracle.point_triangle_distance(p, tris))
    seeds = I.voronoi_seeds(4, 6, (14, 14, 14))
    ms = oracle.tessellate((14, 14, 14), seeds, with_idf=True)
    g = ms.grains[0]
    tr, gr = oracle.gb_triangles(g.phi, g.idf)
    fast = oracle.closest_gb_grains(g.phi, g.idf, 2.5, block=7)
    for z, y, x in np.argwhere(np.abs(g.phi) < 2.5):
        assert fast[z, y, x] == oracle.closest_gb_grain_at((z, y, x), tr, gr)


def test_label_arc_is_the_shortest_covering_interval(oracle):
    """R17: against brute force over every cyclic interval on random
    occupancies (a few cells, runs of them, everything), the arc covers every
    coordinate, no shorter interval does, and among the shortest the one
    whose empty complement starts first is taken."""
    rng = np.random.default_rng(7)
    for n in (1, 2, 5, 9, 16):
        for trial in range(40):
            k = int(rng.integers(1, n + 1))
            coords = rng.choice(n, size=k, replace=False)
            if trial % 7 == 0:
                coords = (int(rng.integers(0, n)) + np.arange(k)) % n    # one run, maybe wrapping
            occ = np.zeros(n, bool)
            occ[coords] = True
            covering = [(s, L) for L in range(1, n + 1) for s in range(n)
                        if all(((c - s) % n) < L for c in coords)]
            best = min(L for _, L in covering)
            start, length = oracle.label_arc(coords, n)
            assert length == best
            assert all(((c - start) % n) < length for c in coords)
            if length < n:
                # the gap left out starts at (start + length) mod n: the first of the longest
                gaps = sorted(((s + L) % n for s, L in covering if L == best))
                assert (start + length) % n == gaps[0]


def test_label_init_of_a_planar_bicrystal_is_exact(oracle):
    """R17 on two slabs (x < 10 and x >= 10 of a periodic 24-cell axis, full
    in y and z): each grain's function is the distance to its two faces
    (x = -0.5 and x = 9.5 for grain 0), +1/2 at the cells next to them, taxicab
    beyond and clamped at eps; the boxes are the slabs grown by the halo, the
    full axes wrapping; the ID-field names the other grain wherever its box
    reaches (-1 beyond: no other function above -eps)."""
    lab = np.zeros((6, 7, 24), dtype=np.int64)
    lab[:, :, 10:] = 1
    ms = oracle.tessellate_labels(lab, 2, eps=7.0, halo=5, with_idf=True)
    g0, g1 = ms.grains
    assert g0.dims == (6, 7, 20) and g0.origin[2] == 19
    assert g1.dims == (6, 7, 24)                       # 14 + 10 cells reach the domain: full
    x = (g0.origin[2] + np.arange(20)) % 24
    d0 = np.minimum(np.abs(x - (-0.5)), np.abs(x - 9.5))
    d0 = np.minimum(d0, np.abs(x - 23.5))
    want0 = np.clip(np.where(x < 10, d0, -d0), -7, 7)
    assert np.array_equal(g0.phi, np.broadcast_to(want0, g0.phi.shape))
    assert np.all(g0.idf == 1)
    x1 = (g1.origin[2] + np.arange(24)) % 24
    in0 = ((x1 - g0.origin[2]) % 24) < g0.dims[2]
    assert np.array_equal(g1.idf, np.broadcast_to(np.where(in0, 0, -1), g1.idf.shape))


def test_label_init_signs_are_the_labels(oracle):
    """R17 on a periodic Voronoi label field: every grain's function is
    positive exactly on its own label cells inside its box and its box holds
    all of them; the ID-field never names the grain itself."""
    shape = (14, 16, 18)
    seeds = I.voronoi_seeds(31, 9, (18, 16, 14))
    lab = oracle.labels_of_tessellation(shape, seeds)
    ms = oracle.tessellate_labels(lab, 9, with_idf=True)
    for g in ms.grains:
        if not g.alive:
            assert not (lab == g.gid).any()
            continue
        pz, py, px = oracle.box_positions(g, shape)
        mine = lab[np.ix_(pz, py, px)] == g.gid
        assert np.array_equal(g.phi > 0, mine)
        assert mine.sum() == (lab == g.gid).sum()
        assert not np.any(g.idf == g.gid)
        assert np.all(np.abs(g.phi) >= 0.5 / np.sqrt(3) - 1e-12)
