"""FP64 CPU oracle of the local level-set grain-growth step.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct
restatement of the method that the CUDA path is checked against.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  It shares no code with the CUDA path; the only
module both use is ``paper_1701_06658_gb300.inputs`` (seeded random numbers).

Source: C. Miessen, N. Velinov, G. Gottstein, L.A. Barrales-Mora, "A highly
efficient 3D level-set grain growth algorithm tailored for ccNUMA
architecture" (arXiv:1701.06658).  Every function cites the section /
equation it restates; equations are numbered in order of appearance:
(1) zero level set, (2) |grad phi| = 1, (7) heat equation, (8) Gaussian
kernel, (9) d(t) = G(t) * d(0), (10) velocity correction, (13) bulk
normalisation, (14)-(15) time map, (16) comparison step, (18) magnetic
energy, (19) magnetic pressure, (20) GB mobility.

Conventions (grid units, h = 1, M_max * gamma_max = 1):
  * arrays are indexed (z, y, x) (x fastest); a domain has shape (Nz, Ny, Nx);
    Nz == 1 is a 2D domain, whose z axis is never convolved, searched or
    resized;
  * the domain is periodic; a grain owns a box with origin o (in [0, N)) and
    dims n <= N per axis; box cell l sits at global cell (o + l) mod N;
  * an axis with n == N is "full": it wraps onto itself;
  * outside its box a grain's function is -eps (Fig. 1 caption: "outside it
    was restricted to eps = -7h").

Pins (tests/test_oracle_pins.py) tie every function here to something other
than itself.  Parity unpinned: the evolution of many grains over many steps
(``run``) beyond what those pins fix -- its laws (sphere, circle, von
Neumann-Mullins), invariants (no voids or overlaps) and stationary cases --
has no independent reference; there the device path is judged against this
module alone.

Readings of points where the paper is silent or garbled (each named in the
code where it applies):
  R1 Eq. (8) prints (4 pi t)^(-1/D) exp(-|x|^2 / 4 pi); we use the heat kernel
     of Eq. (7), exp(-|x|^2 / (4 t)), sampled at integer offsets |k| <= R,
     normalised to sum 1 and applied separably.
  R2 values are clamped to [-eps, eps] after the predictor and redistancing.
  R3 Eq. (10): phi_p = phi + w (G*phi - phi) + M (e_j - e_i) dt, with the
     pair (i, j) taken per cell from the ID-field of the previous step.  With
     no physics (w = 1, no bulk term) phi_p = G*phi.
  R4 Eq. (16): the max runs over all other grains (-eps outside their boxes);
     all grains compare predicted values of the same step (Jacobi); the
     ID-field is the argmax over grains whose value exceeds -eps, lowest id on
     ties, -1 when none does.
  R5 Sec. 2.1.6 (Zhao's scheme, taxicab metric): a cell whose face neighbour
     (outside the box: -eps) has the opposite sign is a reference cell and
     gets the planar-exact distance s / sqrt(sum_a delta_a^-2), delta_a the
     nearest linear zero crossing along axis a; every other cell gets
     s * min(eps, min over same-sign face neighbours |d| + 1), iterated to the
     fixed point.  sign(0) = -1.
  R6 Sec. 2.1.3 / 3.1 (size-adaptive grids): after every step the box becomes
     the bounding box of {phi > 0} grown by the halo; an axis whose extent
     reaches N becomes full (and keeps its origin if it was full already).
     Values move with their global cell; new cells get -eps.  A grain with no
     positive cell is extinct.
  R7 initial functions (Sec. 2.1.3, "initialized to fulfill Eq. (2)"): the
     minimum over face-adjacent cells of the signed distance to the power
     bisector plane, clamped to [-eps, eps].
  R11 Godunov variant of R5 (the Euclidean first-order update of Zhao's
     fast sweeping, selected instead of the paper's taxicab propagation; Sec.
     6.1 names the metric as the taxicab's weakness): the same reference
     cells and values; every other cell gets the smallest u with
     sum over the axes whose neighbour minimum a_k < u of (u - a_k)^2 = 1,
     capped at eps, iterated (Jacobi) to the fixed point.
  R16 Hartmann variant of R5 (Sec. 2.1.6 names the constrained
     reinitialization of Hartmann, Meinke and Schroeder (J. Comput. Phys. 227,
     2008) as the accurate, ~40x costlier alternative to Zhao's scheme and
     prints only the equation it modifies, Sussman's
     phi_tau + S(phi0) (|grad phi| - 1) = 0): we take their first constrained
     form, phi_tau + S(phi0) (|grad phi| - 1) = beta F, with S(phi0) =
     phi0 / sqrt(phi0^2 + h^2), |grad phi| by Godunov's first-order upwind
     scheme, and F = (phi~ - phi) / h on the cells with a face neighbour of
     the opposite sign in phi0 (outside the box: -eps), where phi~ is the mean
     over those neighbours j of (phi0_i / phi0_j) phi_j -- the value that keeps
     every linearly interpolated zero crossing of phi0 in place; F = 0
     elsewhere.  Forward Euler, dtau = h / 2, beta = 1/2, 20 iterations (the
     band of eps = 7 cells is reached at unit speed), values outside the box
     -eps, every iterate clamped to [-eps, eps].
  R12 grid coarsening (Sec. 4.1, sequential optimizations: the spacing grows
     as the population falls, each function is projected to the coarser grid
     by trilinear interpolation): the same periodic domain on N' < N cells
     per axis, one spacing for all axes (N'/N equal).  Coarse cell i' sits at
     fine index coordinate u = i' N / N' (cell 0 stays in place); its value
     is the trilinear interpolation of the fine values at floor(u) and
     floor(u) + 1 per axis (-eps outside the fine box), times N'/N (distances
     in coarse cells), clamped to [-eps, eps].  The projected function is
     then re-initialised (R5 / R11) on its coarse box -- the projection
     leaves a valid band of only eps N'/N coarse cells -- and the box update
     (R6) follows.  The coarse box of a grain covers every coarse cell whose
     interpolation corners can meet its fine box.  With physics, the ID-field
     the next step's correction reads (R3) is rebuilt on the coarse grid as
     R4's argmax over the other grains of the re-initialised functions.  Time
     and dt stay in grid units (one step's physical time grows with the
     spacing squared).
  R14 size analysis (Sec. 5): rho = <R>^2 / <R^2> and Var(R / <R>) =
     <R^2> / <R>^2 - 1 (= 1 / rho - 1, Eq. (varianz)) from the equivalent
     radii of the grain volumes; Eq. (Rios) with the garbled factor
     nu^(H0/2) read as nu^(H/2) (the only reading under which it is a
     normalised density); the kinetic law is printed as
     <R>^n - <R_0>^n = k t with exponents n = 0.45-0.46, which only makes
     sense as <R> ~ t^n: we fit <R>^(1/n) - <R_0>^(1/n) = k t.
  R15 anisotropy map (Sec. 2.1.4: a grid point takes the energy and mobility
     of the closest point on the grain boundary, found on a marching-cubes
     triangulation; Sec. 4.1 adds junction clustering only as a speed-up):
     the boundary of grain i is the zero level of its box function,
     triangulated by marching tetrahedra (each cell cube split into six
     tetrahedra around its main diagonal, linear interpolation on the edges
     -- the same edge points as marching cubes, without its ambiguous
     cases).  A triangle faces the grain most frequent in the ID-field among
     its tetrahedron's corners with phi_i <= 0 (the lowest id on ties).
     Every cell with |phi_i| < tube adopts the grain of the Euclidean-closest
     triangle; that map replaces R3's per-cell ID-field in Eq. (10)'s
     weights (``Physics.gb_map_tube``).  Box-local: the cubes are those between the box's own cells (a
     full periodic axis is not wrapped; a box with an axis of one cell has
     none, and then the map is the ID-field).
  R17 initialisation from a label field (a tessellation read from a file,
     the paper's input form, Sec. 3.1; the paper gives no rule for it): grain
     i's box is, per axis, the shortest cyclic interval of [0, N) holding
     every label cell of i -- the complement of the longest run of positions
     without one, the first such run counted from 0 on ties -- grown by the
     halo (dims capped at N); its function is R5's re-initialisation of +1/2
     on its label cells and -1/2 on the box's other cells (the zero level on
     the faces between labels, reference cells at 1/2 / sqrt(crossings),
     taxicab distances beyond).  The initial ID-field is, per cell, the other
     grain with the largest function there above -eps (lowest id on ties).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------


def spatial_axes(shape):
    """Axes that carry space: (0, 1, 2) in 3D, (1, 2) in 2D."""
    return (1, 2) if shape[0] == 1 else (0, 1, 2)


@dataclass
class Grain:
    """Grain object of Sec. 3.1: its id, its box Omega_i and its function."""
    gid: int
    origin: tuple            # (oz, oy, ox), each in [0, N)
    phi: np.ndarray          # float64, shape (nz, ny, nx)
    idf: np.ndarray | None = None   # ID-field, int64, same shape (R3/R4)
    alive: bool = True

    @property
    def dims(self):
        return self.phi.shape


def full_axes(grain: Grain, shape):
    return tuple(grain.dims[a] == shape[a] for a in range(3))


def box_positions(grain: Grain, shape):
    """Global cell index along each axis for every local index of the box."""
    return tuple((grain.origin[a] + np.arange(grain.dims[a])) % shape[a] for a in range(3))


def sample(grain: Grain, pos, shape, fill):
    """Values of the grain's function at the outer product of the global
    positions ``pos`` = (pz, py, px); ``fill`` where the box does not reach."""
    loc = []
    inside = []
    for a in range(3):
        l = (pos[a] - grain.origin[a]) % shape[a]
        ok = l < grain.dims[a]
        loc.append(np.where(ok, l, 0))
        inside.append(ok)
    vals = grain.phi[np.ix_(loc[0], loc[1], loc[2])]
    mask = inside[0][:, None, None] & inside[1][None, :, None] & inside[2][None, None, :]
    return np.where(mask, vals, fill), mask


def boxes_intersect(gi: Grain, gj: Grain, shape):
    """True when the two boxes share a cell of the periodic domain."""
    for a in range(3):
        n, oi, ni, oj, nj = shape[a], gi.origin[a], gi.dims[a], gj.origin[a], gj.dims[a]
        if ni == n or nj == n:
            continue
        # j starts inside i's interval, or i starts inside j's interval
        if not ((oj - oi) % n < ni or (oi - oj) % n < nj):
            return False
    return True


def _shift(a, axis, k, wrap, fill):
    """b[x] = a[x + k] along ``axis`` (k = +-1); periodic when ``wrap``."""
    if wrap:
        return np.roll(a, -k, axis=axis)
    b = np.full_like(a, fill)
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if k > 0:
        src[axis] = slice(k, None)
        dst[axis] = slice(None, -k)
    else:
        src[axis] = slice(None, k)
        dst[axis] = slice(-k, None)
    b[tuple(dst)] = a[tuple(src)]
    return b


# --------------------------------------------------------------------------
# predictor: Eqs. (7)-(10), Sec. 2.1.4
# --------------------------------------------------------------------------


def heat_kernel_taps(dt: float, radius: int) -> np.ndarray:
    """1D taps of the heat kernel for time dt (reading R1): G(dt, k) is
    proportional to exp(-k^2 / (4 dt)), |k| <= radius, normalised to sum 1.
    Its second moment is 2 dt (up to truncation), the variance of the
    Green's function of Eq. (7)."""
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-k * k / (4.0 * dt))
    return g / g.sum()


def extend(phi: np.ndarray, full, radius: int, eps: float, axes) -> np.ndarray:
    """Pad the box by ``radius`` cells per spatial axis: periodic copies on a
    full axis, -eps elsewhere (Fig. 1 caption)."""
    out = phi
    for a in axes:
        pad = [(0, 0)] * 3
        pad[a] = (radius, radius)
        if full[a]:
            out = np.pad(out, pad, mode="wrap")
        else:
            out = np.pad(out, pad, mode="constant", constant_values=-eps)
    return out


def convolve(phi: np.ndarray, full, taps: np.ndarray, eps: float, axes) -> np.ndarray:
    """G * phi on the box (Eq. (9)), the 3D (2D) kernel being the outer
    product of ``taps``; applied one axis after the other."""
    radius = (len(taps) - 1) // 2
    c = extend(phi, full, radius, eps, axes)
    for a in axes:
        n = c.shape[a] - 2 * radius
        acc = np.zeros(c.shape[:a] + (n,) + c.shape[a + 1:])
        for t in range(2 * radius + 1):
            sl = [slice(None)] * 3
            sl[a] = slice(t, t + n)
            acc += taps[t] * c[tuple(sl)]
        c = acc
    return c


def predict(grain: Grain, shape, taps, eps, physics=None, dt=1.0) -> np.ndarray:
    """Predictor of Algorithm 1 (Sec. 2.1.4): convolution with the heat
    kernel (Eq. (9)) and, with physics, the velocity correction of Eq. (10)
    (reading R3, or R15 with ``physics.gb_map_tube``).  Clamped to
    [-eps, eps] (reading R2)."""
    axes = spatial_axes(shape)
    c = convolve(grain.phi, full_axes(grain, shape), taps, eps, axes)
    if physics is None:
        phip = c
    else:
        pair_ids = grain.idf
        if physics.gb_map_tube is not None:
            pair_ids = closest_gb_grains(grain.phi, grain.idf, physics.gb_map_tube)   # R15
        w, bulk = physics.blend_terms(grain.gid, pair_ids, dt)
        phip = grain.phi + w * (c - grain.phi) + bulk
    return np.clip(phip, -eps, eps)


# --------------------------------------------------------------------------
# corrector: Eq. (16), Sec. 2.1.5 and the ID-field of Sec. 3.1
# --------------------------------------------------------------------------


def neighbour_max(i: int, grains, phip: dict, shape, eps, candidates=None):
    """max_{j != i} phi_p_j over the cells of box i, and its argmax (R4).

    ``candidates`` restricts j to a superset of the grains whose boxes meet
    box i (the neighbour preselection of Sec. 3.1); it cannot change the
    result because every other grain contributes -eps."""
    gi = grains[i]
    pos = box_positions(gi, shape)
    m = np.full(gi.dims, -eps)
    idm = np.full(gi.dims, -1, dtype=np.int64)
    js = range(len(grains)) if candidates is None else sorted(candidates)
    for j in js:
        gj = grains[j]
        if j == i or not gj.alive:
            continue
        view = Grain(gj.gid, gj.origin, phip[j])
        v, _ = sample(view, pos, shape, -eps)
        better = v > m          # strict: ascending j keeps the lowest id on ties
        m = np.where(better, v, m)
        idm = np.where(better, j, idm)
    return m, idm


def compare(phip_i: np.ndarray, m: np.ndarray) -> np.ndarray:
    """Eq. (16): d_c = (d_p - max_{j != i} d_p_j) / 2."""
    return 0.5 * (phip_i - m)


# --------------------------------------------------------------------------
# re-initialisation: Sec. 2.1.6 (Zhao's fast sweeping, taxicab metric)
# --------------------------------------------------------------------------


def reference_values(phic: np.ndarray, full, eps, axes):
    """Reference cells and their planar-exact distances (reading R5).

    Returns (is_ref, |d_ref|)."""
    pos = phic > 0
    a = np.abs(phic)
    is_ref = np.zeros(phic.shape, dtype=bool)
    inv2 = np.zeros(phic.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        for ax in axes:
            dmin = np.full(phic.shape, np.inf)
            for k in (1, -1):
                nb = _shift(phic, ax, k, full[ax], -eps)
                opp = (nb > 0) != pos
                delta = a / (a + np.abs(nb))
                dmin = np.where(opp, np.minimum(dmin, delta), dmin)
            has = np.isfinite(dmin)
            is_ref |= has
            inv2 = inv2 + np.where(has, 1.0 / (dmin * dmin), 0.0)
        dref = np.where(is_ref, 1.0 / np.sqrt(inv2), 0.0)
    return is_ref, dref


def redistance(phic: np.ndarray, full, eps, axes) -> np.ndarray:
    """Taxicab signed distance to the zero level of phic (reading R5):
    reference values held fixed, d = s * min(eps, min_{same-sign face
    neighbour y} |d(y)| + 1) iterated until nothing changes."""
    pos = phic > 0
    is_ref, dref = reference_values(phic, full, eps, axes)
    mag = np.where(is_ref, dref, eps)
    exists = np.ones(phic.shape, dtype=bool)
    while True:
        cand = np.full(phic.shape, np.inf)
        for ax in axes:
            for k in (1, -1):
                nb_mag = _shift(mag, ax, k, full[ax], np.inf)
                nb_pos = _shift(pos, ax, k, full[ax], False)
                nb_ok = _shift(exists, ax, k, full[ax], False)
                same = nb_ok & (nb_pos == pos)
                cand = np.where(same, np.minimum(cand, nb_mag + 1.0), cand)
        new = np.where(is_ref, dref, np.minimum(eps, cand))
        if np.array_equal(new, mag):
            break
        mag = new
    return np.where(pos, mag, -mag)


def godunov_update(mins) -> np.ndarray:
    """R11: the upwind solution u of sum_k max(u - a_k, 0)^2 = 1 for the
    per-axis neighbour minima a_k (inf where an axis has none): with the a_k
    sorted, u = a_1 + 1 while that is <= a_2, else the root over the two
    smallest while it is <= a_3, else the root over all three."""
    a = np.sort(np.stack(mins), axis=0)
    u = a[0] + 1.0
    if len(mins) >= 2:
        s2 = a[0] + a[1]
        with np.errstate(invalid="ignore"):
            u2 = 0.5 * (s2 + np.sqrt(np.maximum(2.0 - (a[0] - a[1]) ** 2, 0.0)))
        u = np.where(u > a[1], u2, u)
    if len(mins) == 3:
        s3 = a[0] + a[1] + a[2]
        with np.errstate(invalid="ignore"):
            u3 = (s3 + np.sqrt(np.maximum(s3 * s3 - 3.0 * (a[0] ** 2 + a[1] ** 2 + a[2] ** 2 - 1.0), 0.0))) / 3.0
        u = np.where(u > a[2], u3, u)
    return u


def redistance_godunov(phic: np.ndarray, full, eps, axes) -> np.ndarray:
    """Reading R11: Euclidean first-order (Godunov upwind) signed distance to
    the zero level of phic, reference values as in R5 held fixed, the others
    lowered to the fixed point of the update over same-sign face neighbours."""
    pos = phic > 0
    is_ref, dref = reference_values(phic, full, eps, axes)
    mag = np.where(is_ref, dref, eps)
    exists = np.ones(phic.shape, dtype=bool)
    while True:
        mins = []
        for ax in axes:
            m = np.full(phic.shape, np.inf)
            for k in (1, -1):
                nb_mag = _shift(mag, ax, k, full[ax], np.inf)
                nb_pos = _shift(pos, ax, k, full[ax], False)
                nb_ok = _shift(exists, ax, k, full[ax], False)
                m = np.where(nb_ok & (nb_pos == pos), np.minimum(m, nb_mag), m)
            mins.append(m)
        new = np.where(is_ref, dref, np.minimum(mag, np.minimum(eps, godunov_update(mins))))
        if np.array_equal(new, mag):
            break
        mag = new
    return np.where(pos, mag, -mag)


HCR_ITERS = 20      # R16: pseudo-time iterations
HCR_DTAU = 0.5      # R16: pseudo-time step (grid units)
HCR_BETA = 0.5      # R16: weight of the constraint forcing


def hartmann_constraint(phi0: np.ndarray, full, eps, axes):
    """R16: for every cell and face-neighbour direction, whether the neighbour
    has the opposite sign in phi0 (and a non-zero value), and the ratio
    phi0_i / phi0_j that keeps the zero crossing between them in place.
    Returns [(axis, k, use, ratio)], count."""
    pos0 = phi0 > 0
    terms, count = [], np.zeros(phi0.shape)
    for ax in axes:
        for k in (1, -1):
            nb0 = _shift(phi0, ax, k, full[ax], -eps)
            use = ((nb0 > 0) != pos0) & (nb0 != 0.0)
            with np.errstate(divide="ignore", invalid="ignore"):
                ratio = np.where(use, phi0 / np.where(use, nb0, 1.0), 0.0)
            terms.append((ax, k, use, ratio))
            count += use
    return terms, count


def godunov_gradient_norm(phi: np.ndarray, s0: np.ndarray, full, eps, axes) -> np.ndarray:
    """|grad phi| by Godunov's upwind scheme for phi_tau + S (|grad phi| - 1)
    = 0 (Sussman et al.'s reinitialization equation): per axis with the
    backward and forward differences a = phi_i - phi_{i-1}, b = phi_{i+1} -
    phi_i, the term max(max(a, 0)^2, min(b, 0)^2) where S > 0 and
    max(min(a, 0)^2, max(b, 0)^2) where S <= 0; -eps outside the box."""
    g2 = np.zeros(phi.shape)
    for ax in axes:
        a = phi - _shift(phi, ax, -1, full[ax], -eps)
        b = _shift(phi, ax, 1, full[ax], -eps) - phi
        gp = np.maximum(np.maximum(a, 0.0) ** 2, np.minimum(b, 0.0) ** 2)
        gn = np.maximum(np.minimum(a, 0.0) ** 2, np.maximum(b, 0.0) ** 2)
        g2 = g2 + np.where(s0 > 0, gp, gn)
    return np.sqrt(g2)


def redistance_hartmann(phic: np.ndarray, full, eps, axes, iters: int = HCR_ITERS, dtau: float = HCR_DTAU,
                        beta: float = HCR_BETA) -> np.ndarray:
    """Reading R16: Hartmann et al.'s constrained reinitialization, first form:
    forward-Euler steps of phi_tau + S(phi0) (|grad phi| - 1) = beta F from
    phi0 = phic, F = (phi~ - phi) / h on the cells next to the zero level
    (phi~ = mean over their opposite-sign neighbours j of (phi0_i / phi0_j)
    phi_j), clamped to [-eps, eps] after every step."""
    phi0 = np.asarray(phic, dtype=np.float64)
    s0 = phi0 / np.sqrt(phi0 * phi0 + 1.0)
    terms, count = hartmann_constraint(phi0, full, eps, axes)
    gamma = count > 0
    phi = phi0.copy()
    for _ in range(iters):
        grad = godunov_gradient_norm(phi, s0, full, eps, axes)
        cons = np.zeros(phi.shape)
        for ax, k, use, ratio in terms:
            cons = cons + np.where(use, ratio * _shift(phi, ax, k, full[ax], -eps), 0.0)
        force = np.where(gamma, cons / np.maximum(count, 1.0) - phi, 0.0)
        phi = np.clip(phi - dtau * s0 * (grad - 1.0) + dtau * beta * force, -eps, eps)
    return phi


def redistancer(name: str):
    """The re-initialisation of a scheme name: "taxicab" (R5), "godunov"
    (R11) or "hartmann" (R16)."""
    return {"taxicab": redistance, "godunov": redistance_godunov, "hartmann": redistance_hartmann}[name]


# --------------------------------------------------------------------------
# box update: Secs. 2.1.3 and 3.1 (size-adaptive local grids)
# --------------------------------------------------------------------------


def box_update(grain: Grain, shape, halo: int, eps: float) -> Grain:
    """New box = bbox{phi > 0} grown by ``halo`` (reading R6)."""
    pos = grain.phi > 0
    if not pos.any():
        return Grain(grain.gid, grain.origin, grain.phi, grain.idf, alive=False)
    axes = spatial_axes(shape)
    origin = list(grain.origin)
    dims = list(grain.dims)
    for a in axes:
        other = tuple(b for b in range(3) if b != a)
        occ = np.nonzero(pos.any(axis=other))[0]
        lmin, lmax = int(occ[0]), int(occ[-1])
        n = lmax - lmin + 1 + 2 * halo
        was_full = grain.dims[a] == shape[a]
        if n >= shape[a]:
            dims[a] = shape[a]
            origin[a] = grain.origin[a] if was_full else (grain.origin[a] + lmin - halo) % shape[a]
        else:
            dims[a] = n
            origin[a] = (grain.origin[a] + lmin - halo) % shape[a]
    new = Grain(grain.gid, tuple(origin), np.zeros(tuple(dims)))
    pos_new = box_positions(new, shape)
    new.phi, _ = sample(grain, pos_new, shape, -eps)
    if grain.idf is not None:
        idv = Grain(grain.gid, grain.origin, grain.idf)
        new.idf, _ = sample(idv, pos_new, shape, -1)
        new.idf = new.idf.astype(np.int64)
    return new


# --------------------------------------------------------------------------
# physics of the velocity correction: Eqs. (10), (13)-(15), (18)-(20), Sec. 4.3
# --------------------------------------------------------------------------


def _qmul(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def cubic_symmetry_quaternions() -> np.ndarray:
    """The 24 proper rotations of the cube as unit quaternions (w, x, y, z):
    identity, 3 half turns about the axes, 6 quarter turns about the axes,
    8 third turns about the body diagonals, 6 half turns about the face
    diagonals."""
    c = 1.0 / math.sqrt(2.0)
    ops = [(1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1)]
    for ax in range(3):
        for s in (1, -1):
            v = [c, 0.0, 0.0, 0.0]
            v[1 + ax] = s * c
            ops.append(tuple(v))
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                ops.append((0.5, 0.5 * sx, 0.5 * sy, 0.5 * sz))
    for (p, q) in ((1, 2), (1, 3), (2, 3)):
        for s in (1, -1):
            v = [0.0, 0.0, 0.0, 0.0]
            v[p] = c
            v[q] = s * c
            ops.append(tuple(v))
    return np.array(ops, dtype=np.float64)


_CUBIC = cubic_symmetry_quaternions()


def disorientation_cubic(qa, qb) -> float:
    """Smallest rotation angle (radians) taking crystal a to crystal b under
    cubic symmetry: 2 acos(max_k |w(conj(qa) qb S_k)|)."""
    qa = np.asarray(qa, dtype=np.float64)
    conj = qa * np.array([1.0, -1.0, -1.0, -1.0])
    dq = _qmul(conj, np.asarray(qb, dtype=np.float64))
    best = max(abs(_qmul(dq, s)[0]) for s in _CUBIC)
    return 2.0 * math.acos(min(1.0, best))


def read_shockley(theta: float, theta_max: float) -> float:
    """Normalised Read-Shockley energy (Sec. 4.3): (t)(1 - ln t) with
    t = theta / theta_max below theta_max, 1 above."""
    if theta >= theta_max:
        return 1.0
    if theta <= 0.0:
        return 0.0
    t = theta / theta_max
    return t * (1.0 - math.log(t))


def mobility_step(theta: float, theta_max: float, low: float) -> float:
    """Normalised mobility: ``low`` below theta_max, 1 above."""
    return low if theta < theta_max else 1.0


def mobility_eq20(theta: float) -> float:
    """Eq. (20): mu = 1 - 0.99 exp(-5 (theta / 15 deg)^9), as printed (its
    rise lies between 10 and 15 degrees, where the prose says 8 to 10)."""
    return 1.0 - 0.99 * math.exp(-5.0 * (theta / math.radians(15.0)) ** 9)


MU0 = 4.0e-7 * math.pi


def magnetic_energy_density(b_tesla: float, dchi: float, cos2: float) -> float:
    """Eqs. (18)-(19): orientation-dependent part of mu0 H^2 chi / 2 with
    H = B / mu0, chi = chi_perp + dchi cos^2(theta); chi_perp cancels in
    every difference, so E = B^2 dchi cos^2 / (2 mu0) in J/m^3."""
    return b_tesla * b_tesla * dchi * cos2 / (2.0 * MU0)


def c_axis(q) -> np.ndarray:
    """Crystal [001] direction rotated by the unit quaternion q = (w, x, y, z)."""
    w, x, y, z = q
    return np.array([2.0 * (x * z + w * y), 2.0 * (y * z - w * x), 1.0 - 2.0 * (x * x + y * y)])


@dataclass
class Physics:
    """Per-pair weights and per-grain bulk energies of Eq. (10).

    weight(i, j) -> (w_ij, M_ij): w = M* gamma* in (0, 1] scales the
    curvature flow, M* in (0, 1] the bulk term.  ``energy[i]`` is the bulk
    energy of grain i in grid units (E_i h / gamma_max, Eq. (13)).
    ``gb_map_tube``: None takes the pair per cell from the ID-field (R3); a
    tube width takes it from the closest grain-boundary point instead (R15)
    for the cells with |phi| below it."""
    weight: callable
    energy: np.ndarray
    _cache: dict = field(default_factory=dict)
    gb_map_tube: float | None = None

    def pair(self, i, j):
        key = (i, j)
        if key not in self._cache:
            self._cache[key] = self.weight(i, j)
        return self._cache[key]

    def blend_terms(self, gid, idf, dt):
        """Per-cell w and bulk = M (e_j - e_i) dt for pair (gid, ID(x));
        w = 1 and bulk = 0 where the ID-field is -1."""
        w = np.ones(idf.shape)
        bulk = np.zeros(idf.shape)
        for j in np.unique(idf):
            if j < 0:
                continue
            wij, mij = self.pair(gid, int(j))
            sel = idf == j
            w[sel] = wij
            bulk[sel] = mij * (self.energy[int(j)] - self.energy[gid]) * dt
        return w, bulk


def isotropic_physics(energy) -> Physics:
    """w = M = 1 for every pair, per-grain bulk energies (Sec. 4.1 / 4.3)."""
    return Physics(weight=lambda i, j: (1.0, 1.0), energy=np.asarray(energy, dtype=np.float64))


def read_shockley_physics(quats, theta_max_deg=15.0, mob_low=0.1, mobility="step",
                          w_floor=1e-3) -> Physics:
    """Read-Shockley energy and low/high-angle mobility per pair (Sec. 4.3),
    cubic disorientation; w = max(w_floor, M* gamma*)."""
    qs = np.asarray(quats, dtype=np.float64)
    tm = math.radians(theta_max_deg)

    def weight(i, j):
        th = disorientation_cubic(qs[i], qs[j])
        m = mobility_step(th, tm, mob_low) if mobility == "step" else mobility_eq20(th)
        return max(w_floor, m * read_shockley(th, tm)), m
    return Physics(weight=weight, energy=np.zeros(len(qs)))


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------


@dataclass
class Microstructure:
    shape: tuple                 # (Nz, Ny, Nx)
    grains: list
    eps: float = 7.0
    halo: int = 5
    radius: int = 5
    physics: Physics | None = None
    time: float = 0.0
    redist: str = "taxicab"      # R5, or "godunov" (R11), or "hartmann" (R16)


def box_candidates(ms: Microstructure):
    """Grains whose boxes meet each box (Sec. 3.1's neighbour preselection)."""
    alive = [g for g in ms.grains if g.alive]
    out = {g.gid: set() for g in ms.grains}
    for a_i, gi in enumerate(alive):
        for gj in alive[a_i + 1:]:
            if boxes_intersect(gi, gj, ms.shape):
                out[gi.gid].add(gj.gid)
                out[gj.gid].add(gi.gid)
    return out


@dataclass
class StepParts:
    """Intermediate results of one step, per grain id."""
    phip: dict
    m: dict
    idm: dict
    phic: dict
    phi: dict


def step_parts(ms: Microstructure, dt: float, brute_force: bool = False) -> StepParts:
    """Predictor, corrector and re-initialisation of Algorithm 1 on the
    current boxes, without the box update."""
    taps = heat_kernel_taps(dt, ms.radius)
    axes = spatial_axes(ms.shape)
    phip = {}
    for g in ms.grains:
        if g.alive:
            phip[g.gid] = predict(g, ms.shape, taps, ms.eps, ms.physics, dt)
    cand = None if brute_force else box_candidates(ms)
    parts = StepParts(phip, {}, {}, {}, {})
    for g in ms.grains:
        if not g.alive:
            continue
        m, idm = neighbour_max(g.gid, ms.grains, phip, ms.shape, ms.eps,
                               None if cand is None else cand[g.gid])
        parts.m[g.gid] = m
        parts.idm[g.gid] = idm
        parts.phic[g.gid] = compare(phip[g.gid], m)
        redist = redistancer(ms.redist)
        parts.phi[g.gid] = np.clip(redist(parts.phic[g.gid], full_axes(g, ms.shape), ms.eps, axes),
                                   -ms.eps, ms.eps)
    return parts


def step(ms: Microstructure, dt: float, brute_force: bool = False) -> Microstructure:
    """One pass of Algorithm 1's loop body plus the box update (R6)."""
    parts = step_parts(ms, dt, brute_force)
    grains = []
    for g in ms.grains:
        if not g.alive:
            grains.append(g)
            continue
        idf = parts.idm[g.gid] if ms.physics is not None else None
        upd = Grain(g.gid, g.origin, parts.phi[g.gid], idf)
        grains.append(box_update(upd, ms.shape, ms.halo, ms.eps))
    return Microstructure(ms.shape, grains, ms.eps, ms.halo, ms.radius, ms.physics, ms.time + dt, ms.redist)


def run(ms: Microstructure, n: int, dt: float) -> Microstructure:
    for _ in range(n):
        ms = step(ms, dt)
    return ms


# --------------------------------------------------------------------------
# grid coarsening: Sec. 4.1 (reading R12)
# --------------------------------------------------------------------------


def coarse_axis(o: int, n: int, N: int, N2: int):
    """Origin and extent on a coarse axis of N2 cells of the box [o, o + n) of
    a fine axis of N cells: every coarse cell i' with a fine interpolation
    corner floor(u) or floor(u) + 1 (u = i' N / N2) in the box, i.e.
    (o - 1) N2 / N <= i' <= (o + n - 1) N2 / N, lies in [floor((o - 1) N2 / N),
    ceil((o + n) N2 / N)] (R12)."""
    if n >= N:
        return (o * N2) // N, N2
    lo = ((o - 1) * N2) // N
    hi = -((-(o + n) * N2) // N)
    n2 = hi - lo + 1
    if n2 >= N2:
        return lo % N2, N2
    return lo % N2, n2


def coarse_project(grain: Grain, shape, shape2, eps: float) -> Grain:
    """The grain's function on its coarse box (R12), before re-initialisation:
    trilinear interpolation of the fine values (-eps outside the fine box) at
    u = i' N / N' per axis, times N' / N, clamped to [-eps, eps]."""
    origin2, dims2 = [], []
    for a in range(3):
        o2, n2 = coarse_axis(grain.origin[a], grain.dims[a], shape[a], shape2[a])
        origin2.append(o2)
        dims2.append(n2)
    pos2 = [(origin2[a] + np.arange(dims2[a])) % shape2[a] for a in range(3)]
    fl, w = [], []
    for a in range(3):
        num = pos2[a] * shape[a]
        fl.append(num // shape2[a])
        w.append((num % shape2[a]) / shape2[a])
    val = np.zeros(tuple(dims2))
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                c = (cz, cy, cx)
                pos = tuple((fl[a] + c[a]) % shape[a] for a in range(3))
                v, _ = sample(grain, pos, shape, -eps)
                wt = [w[a] if c[a] else 1.0 - w[a] for a in range(3)]
                val += wt[0][:, None, None] * wt[1][None, :, None] * wt[2][None, None, :] * v
    scale = shape2[2] / shape[2]
    return Grain(grain.gid, tuple(origin2), np.clip(scale * val, -eps, eps))


def coarsen(ms: Microstructure, shape2) -> Microstructure:
    """Every grain projected onto the coarser grid ``shape2`` of the same
    periodic 3D domain, re-initialised and box-updated (R12)."""
    shape2 = tuple(int(v) for v in shape2)
    if any(ms.shape[a] < 2 for a in range(3)):
        raise ValueError("grid coarsening is defined on 3D domains")
    if any(shape2[a] * ms.shape[2] != shape2[2] * ms.shape[a] for a in range(3)):
        raise ValueError("one spacing for all axes: N'/N must be equal")
    if any(not 1 <= shape2[a] <= ms.shape[a] for a in range(3)):
        raise ValueError("coarser grid expected")
    axes = spatial_axes(shape2)
    redist = redistancer(ms.redist)
    coarse = []
    for g in ms.grains:
        if not g.alive:
            coarse.append(Grain(g.gid, g.origin, g.phi, None, alive=False))
            continue
        p = coarse_project(g, ms.shape, shape2, ms.eps)
        p.phi = np.clip(redist(p.phi, full_axes(p, shape2), ms.eps, axes), -ms.eps, ms.eps)
        coarse.append(p)
    if ms.physics is not None:
        cms = Microstructure(shape2, coarse, ms.eps, ms.halo, ms.radius, ms.physics, ms.time, ms.redist)
        cand = box_candidates(cms)
        phis = {g.gid: g.phi for g in coarse if g.alive}
        for g in coarse:
            if g.alive:
                _, g.idf = neighbour_max(g.gid, coarse, phis, shape2, ms.eps, cand[g.gid])
    grains = [box_update(g, shape2, ms.halo, ms.eps) if g.alive else g for g in coarse]
    return Microstructure(shape2, grains, ms.eps, ms.halo, ms.radius, ms.physics, ms.time, ms.redist)


# --------------------------------------------------------------------------
# outputs
# --------------------------------------------------------------------------


def owner_map(ms: Microstructure) -> np.ndarray:
    """owner(x) = argmax_i phi_i(x) over the boxes that cover x, lowest id on
    ties, -1 where no box covers x."""
    Nz, Ny, Nx = ms.shape
    best = np.full(ms.shape, -np.inf)
    own = np.full(ms.shape, -1, dtype=np.int64)
    allpos = (np.arange(Nz), np.arange(Ny), np.arange(Nx))
    for g in ms.grains:
        if not g.alive:
            continue
        v, _ = sample(g, allpos, ms.shape, -np.inf)
        better = v > best
        best = np.where(better, v, best)
        own = np.where(better, g.gid, own)
    return own


def volumes(ms: Microstructure) -> np.ndarray:
    """V_i = sum_x H(phi_i(x)), H(phi) = clamp(phi + 1/2, 0, 1) (a unit ramp
    across the zero level); 0 for extinct grains."""
    out = np.zeros(len(ms.grains))
    for g in ms.grains:
        if g.alive:
            out[g.gid] = float(np.clip(g.phi + 0.5, 0.0, 1.0).sum())
    return out


def voxel_counts(ms: Microstructure) -> np.ndarray:
    own = owner_map(ms)
    return np.bincount(own[own >= 0].ravel(), minlength=len(ms.grains))


# --------------------------------------------------------------------------
# initial microstructure: Sec. 2.1.3 (tessellation S, local grids Omega_i)
# --------------------------------------------------------------------------


def power_distance(cells_xyz: np.ndarray, s, w, n_xyz) -> np.ndarray:
    """|x - s|^2 - w with the minimum-image displacement per axis:
    d = x - s; d = d - N rint(d / N); (dx^2 + dy^2) + dz^2 - w."""
    d = []
    for a in range(3):
        da = cells_xyz[..., a] - s[a]
        da = da - n_xyz[a] * np.rint(da / n_xyz[a])
        d.append(da)
    r = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
    return r - w if w is not None else r


def labels_at(cells_xyz: np.ndarray, seeds, weights, n_xyz) -> np.ndarray:
    """Voronoi (power) label of each cell: argmin_i of power_distance, lowest
    id on ties."""
    best = np.full(cells_xyz.shape[:-1], np.inf)
    lab = np.full(cells_xyz.shape[:-1], -1, dtype=np.int64)
    for i in range(len(seeds)):
        d = power_distance(cells_xyz, seeds[i], None if weights is None else weights[i], n_xyz)
        better = d < best
        best = np.where(better, d, best)
        lab = np.where(better, i, lab)
    return lab


def domain_cells(shape) -> np.ndarray:
    """Integer cell coordinates (x, y, z) of the whole domain, shape (Nz, Ny, Nx, 3)."""
    Nz, Ny, Nx = shape
    z, y, x = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    return np.stack([x, y, z], axis=-1).astype(np.float64)


def face_neighbours(labels: np.ndarray, n_grains: int):
    """Nb(i): grains whose cells touch grain i's cells across a face (periodic)."""
    nb = [set() for _ in range(n_grains)]
    axes = spatial_axes(labels.shape)
    for a in axes:
        other = np.roll(labels, -1, axis=a)
        diff = labels != other
        for p, q in set(zip(labels[diff].ravel().tolist(), other[diff].ravel().tolist())):
            nb[p].add(q)
            nb[q].add(p)
    return nb


def minimum_image_offset(x: np.ndarray, r: int, n: int) -> np.ndarray:
    """Integer offset e of cell x from cell r on a ring of n cells, chosen in
    (-n/2, n/2] for even n ([-(n-1)/2, (n-1)/2] for odd n)."""
    e = (x - r) % n
    return np.where(e > n // 2, e - n, e)


def initial_box(cells_xyz_int: np.ndarray, seed_xyz, n_xyz, halo: int):
    """Box of one grain: bbox of its label cells (offsets from the rounded
    seed by minimum image) grown by ``halo``; returns origin (z, y, x) and
    dims (z, y, x)."""
    origin = [0, 0, 0]
    dims = [1, 1, 1]
    for a in range(3):
        n = int(n_xyz[a])
        if n == 1:
            continue
        r = int(np.rint(seed_xyz[a])) % n
        e = minimum_image_offset(cells_xyz_int[:, a], r, n)
        lo, hi = int(e.min()), int(e.max())
        ext = hi - lo + 1 + 2 * halo
        za = 2 - a   # (z, y, x) index of axis a of (x, y, z)
        dims[za] = min(ext, n)
        origin[za] = (r + lo - halo) % n
    return tuple(origin), tuple(dims)


def bisector_sdf(pos_xyz: np.ndarray, i: int, nbs, seeds, weights, n_xyz, eps):
    """Reading R7: phi_i(x) = clamp(min_{j in Nb(i)} ((|b|^2 - w_j) - (|a|^2 - w_i))
    / (2 |b - a|), -eps, eps), a = x - s_i, b = x - s_j (minimum images), and the
    minimising j (lowest id on ties; -1 when Nb(i) is empty)."""
    def disp(s):
        out = []
        for a in range(3):
            d = pos_xyz[..., a] - s[a]
            out.append(d - n_xyz[a] * np.rint(d / n_xyz[a]))
        return out
    a_ = disp(seeds[i])
    wi = 0.0 if weights is None else weights[i]
    pa = (a_[0] * a_[0] + a_[1] * a_[1]) + a_[2] * a_[2] - wi
    best = np.full(pos_xyz.shape[:-1], np.inf)
    arg = np.full(pos_xyz.shape[:-1], -1, dtype=np.int64)
    for j in sorted(nbs):
        b_ = disp(seeds[j])
        wj = 0.0 if weights is None else weights[j]
        pb = (b_[0] * b_[0] + b_[1] * b_[1]) + b_[2] * b_[2] - wj
        dx, dy, dz = b_[0] - a_[0], b_[1] - a_[1], b_[2] - a_[2]
        den = 2.0 * np.sqrt((dx * dx + dy * dy) + dz * dz)
        v = (pb - pa) / den
        better = v < best
        best = np.where(better, v, best)
        arg = np.where(better, j, arg)
    best = np.where(np.isfinite(best), best, eps)
    return np.clip(best, -eps, eps), arg


def tessellate(shape, seeds, weights=None, eps=7.0, halo=5, radius=5, physics=None,
               with_idf=False) -> Microstructure:
    """Initialisation of Algorithm 1: one grain per (power) Voronoi cell of
    the seeds, its box (R6's rule applied to the label cells) and its
    initial function (R7).  Grains with no cell are extinct from the start."""
    Nz, Ny, Nx = shape
    n_xyz = (Nx, Ny, Nz)
    seeds = np.asarray(seeds, dtype=np.float64)
    cells = domain_cells(shape)
    lab = labels_at(cells, seeds, weights, n_xyz)
    G = len(seeds)
    nbs = face_neighbours(lab, G)
    grains = []
    for i in range(G):
        sel = lab == i
        if not sel.any():
            grains.append(Grain(i, (0, 0, 0), np.full((1, 1, 1), -eps), None, alive=False))
            continue
        pts = cells[sel].astype(np.int64)
        origin, dims = initial_box(pts, seeds[i], n_xyz, halo)
        g = Grain(i, origin, np.zeros(dims))
        pz, py, px = box_positions(g, shape)
        z, y, x = np.meshgrid(pz, py, px, indexing="ij")
        pos = np.stack([x, y, z], axis=-1).astype(np.float64)
        g.phi, arg = bisector_sdf(pos, i, nbs[i], seeds, weights, n_xyz, eps)
        if with_idf or physics is not None:
            g.idf = arg
        grains.append(g)
    return Microstructure(tuple(shape), grains, eps, halo, radius, physics)


def labels_of_tessellation(shape, seeds, weights=None) -> np.ndarray:
    Nz, Ny, Nx = shape
    return labels_at(domain_cells(shape), np.asarray(seeds, dtype=np.float64), weights, (Nx, Ny, Nz))


def label_arc(coords, n: int):
    """Reading R17: the shortest cyclic interval of [0, n) that holds every
    coordinate in ``coords`` -- the complement of the longest run of
    positions holding none (the first such run counted from 0 on ties);
    returns (start, length)."""
    occ = np.zeros(n, dtype=bool)
    occ[np.asarray(coords, dtype=np.int64) % n] = True
    if occ.all():
        return 0, n
    best_start, best_len = 0, -1
    for s in range(n):
        if occ[s] or not occ[(s - 1) % n]:
            continue                               # not the first position of an empty run
        length = 0
        while not occ[(s + length) % n]:
            length += 1
        if length > best_len:
            best_start, best_len = s, length
    return (best_start + best_len) % n, n - best_len


def label_box(cells_zyx: np.ndarray, shape, halo: int):
    """Reading R17: per axis the label arc of the grain's cells grown by the
    halo (dims capped at the domain); returns origin and dims (z, y, x)."""
    origin, dims = [0, 0, 0], [1, 1, 1]
    for a in range(3):
        n = int(shape[a])
        if n == 1:
            continue
        start, length = label_arc(cells_zyx[:, a], n)
        dims[a] = min(length + 2 * halo, n)
        origin[a] = (start - halo) % n
    return tuple(origin), tuple(dims)


def tessellate_labels(labels: np.ndarray, n_grains: int, eps=7.0, halo=5, radius=5, physics=None,
                      with_idf=False, redist: str = "taxicab") -> Microstructure:
    """Initialisation from a label field (reading R17): grain i (label i) on
    its label box, its function the re-initialisation (R5, or the scheme
    named by ``redist``: R11, R16) of +1/2 on its label cells and -1/2
    elsewhere in the box; grains without a cell are extinct.  With physics
    (or with_idf), the ID-field of every box cell is the other grain whose
    function is largest there above -eps."""
    labels = np.asarray(labels)
    shape = labels.shape
    axes = spatial_axes(shape)
    grains = []
    for i in range(n_grains):
        sel = labels == i
        if not sel.any():
            grains.append(Grain(i, (0, 0, 0), np.full((1, 1, 1), -eps), None, alive=False))
            continue
        origin, dims = label_box(np.argwhere(sel), shape, halo)
        g = Grain(i, origin, np.zeros(dims))
        pz, py, px = box_positions(g, shape)
        mine = labels[np.ix_(pz, py, px)] == i
        g.phi = redistancer(redist)(np.where(mine, 0.5, -0.5), full_axes(g, shape), eps, axes)
        grains.append(g)
    if with_idf or physics is not None:
        phis = {g.gid: g.phi for g in grains if g.alive}
        for g in grains:
            if g.alive:
                _, g.idf = neighbour_max(g.gid, grains, phis, shape, eps)
    return Microstructure(tuple(shape), grains, eps, halo, radius, physics, redist=redist)


def single_grain_state(shape, phi_fn, eps=7.0, halo=5, radius=5):
    """Two-grain state for analytic tests: grain 0 has phi = clamp(phi_fn(x), +-eps)
    on the bbox of its positive set grown by the halo; grain 1 is the
    complement (-phi_fn) on the whole domain.  ``phi_fn`` maps (z, y, x) index
    grids to signed distances."""
    Nz, Ny, Nx = shape
    z, y, x = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    d = phi_fn(z.astype(np.float64), y.astype(np.float64), x.astype(np.float64))
    full = Grain(0, (0, 0, 0), np.clip(d, -eps, eps))
    g0 = box_update(full, shape, halo, eps)
    g1 = Grain(1, (0, 0, 0), np.clip(-d, -eps, eps))
    return Microstructure(tuple(shape), [g0, g1], eps, halo, radius)


# --------------------------------------------------------------------------
# grain statistics: Sec. 5 (mean radius, normalised grain size distribution)
# --------------------------------------------------------------------------


def grain_statistics(vol: np.ndarray, dim: int, n_bins: int, r_max: float) -> dict:
    """Statistics of the alive grains (V > 0) from their volumes: the
    equivalent radius R = (3 V / 4 pi)^(1/3) (3D) or (V / pi)^(1/2) (2D), its
    mean and root mean square, the largest R, and the distribution of R / <R>
    as fractions of the alive grains in n_bins equal bins over [0, r_max)
    (the rest in `overflow`): the quantities of the paper's size analysis."""
    v = vol[vol > 0]
    r = (3.0 * v / (4.0 * math.pi)) ** (1.0 / 3.0) if dim == 3 else np.sqrt(v / math.pi)
    n = r.size
    out = {"alive": n, "mean_volume": 0.0, "mean_radius": 0.0, "rms_radius": 0.0, "max_radius": 0.0,
           "overflow": 0.0, "rho": 0.0, "var_z": 0.0, "hist": np.zeros(n_bins)}
    if n == 0:
        return out
    mean = r.mean()
    rel = r / mean
    k = np.floor(rel / r_max * n_bins).astype(np.int64)
    for b in k[k < n_bins]:
        out["hist"][b] += 1.0
    msq = (r * r).mean()
    out.update(mean_volume=v.mean(), mean_radius=mean, rms_radius=math.sqrt(msq), max_radius=r.max(),
               overflow=float((k >= n_bins).sum()) / n,
               rho=mean * mean / msq,                  # Sec. 5: rho = <R>^2 / <R^2>
               var_z=msq / (mean * mean) - 1.0)        # Eq. (varianz): Var(R / <R>) = 1 / rho - 1
    out["hist"] /= n
    return out



# --------------------------------------------------------------------------
# size distributions and kinetics of the size analysis (Sec. 5, reading R14)
# --------------------------------------------------------------------------


def rios_pdf(z, nu: float, rho: float, H: float = 3.0):
    """Eq. (Rios): Rios' distribution of z = R / <R> with H = 3, reading the
    garbled factor nu^(H0/2) as nu^(H/2), the reading under which p
    integrates to 1 (R14).  Valid for 0 < nu < 4."""
    z = np.asarray(z, dtype=np.float64)
    s = math.sqrt(4.0 * nu - nu * nu)
    base = rho * rho * z * z - nu * rho * z + nu
    ang = np.arctan((2.0 * rho * z - nu) / s) + math.atan(nu / s)
    return z * rho * rho * H * nu ** (H / 2.0) / base ** (1.0 + H / 2.0) * np.exp(-H * nu / s * ang)


def hillert_pdf(z):
    """Hillert's 3D distribution written in z = R / <R>: with u = R / R_cr =
    rho z and rho = 8/9, P(u) = (2e)^3 3u / (2 - u)^5 exp(-6 / (2 - u)) for
    u < 2, so p(z) = rho P(rho z) (the nu -> 4 limit of Eq. (Rios))."""
    z = np.asarray(z, dtype=np.float64)
    rho = 8.0 / 9.0
    u = rho * z
    inside = u < 2.0
    uu = np.where(inside, u, 0.0)
    P = (2.0 * math.e) ** 3 * 3.0 * uu / (2.0 - uu) ** 5 * np.exp(-6.0 / (2.0 - uu))
    return np.where(inside, rho * P, 0.0)


def fit_rios_nu(hist: np.ndarray, r_max: float, rho: float) -> float:
    """nu of Eq. (Rios) closest (least squares over the bins' centres) to a
    measured distribution of R / <R> given as fractions per bin of
    [0, r_max), with the measured rho (Sec. 5 fits nu and rho this way)."""
    from scipy.optimize import minimize_scalar
    n = len(hist)
    w = r_max / n
    zc = (np.arange(n) + 0.5) * w
    dens = np.asarray(hist, dtype=np.float64) / w
    res = minimize_scalar(lambda nu: float(((rios_pdf(zc, nu, rho) - dens) ** 2).sum()),
                          bounds=(1e-3, 4.0 - 1e-6), method="bounded", options={"xatol": 1e-9})
    return float(res.x)


def fit_growth_exponent(t: np.ndarray, mean_r: np.ndarray):
    """Kinetic exponent of Sec. 5 (R14): <R> ~ t^n, fitted in the printed law's
    form <R>^(1/n) - <R_0>^(1/n) = k t (parabolic growth: n = 1/2) by least
    squares over n, with k the least-squares slope through the origin for
    each n and <R_0> the first sample.  Returns (n, k)."""
    from scipy.optimize import minimize_scalar
    t = np.asarray(t, dtype=np.float64)
    r = np.asarray(mean_r, dtype=np.float64)
    dt = t - t[0]

    def cost(n):
        y = r ** (1.0 / n) - r[0] ** (1.0 / n)
        k = float((dt * y).sum() / (dt * dt).sum())
        return float(((y - k * dt) ** 2).sum() / (y * y).sum()), k

    res = minimize_scalar(lambda n: cost(n)[0], bounds=(0.05, 2.0), method="bounded", options={"xatol": 1e-10})
    return float(res.x), cost(res.x)[1]


def texture_shares(vol: np.ndarray, grain_class: np.ndarray, n_classes: int) -> np.ndarray:
    """Volume fraction of each grain class (Sec. 5.3's texture components):
    the class's summed volume over all grains' volume; grains of a class
    outside [0, n_classes) count in the total only."""
    vol = np.asarray(vol, dtype=np.float64)
    out = np.zeros(n_classes)
    for v, c in zip(vol, grain_class):
        if 0 <= c < n_classes:
            out[c] += v
    tot = vol[vol > 0].sum()
    return out / tot if tot > 0 else out


# --------------------------------------------------------------------------
# anisotropy map: Secs. 2.1.4 and 4.1, the closest grain-boundary point (R15)
# --------------------------------------------------------------------------

# the six tetrahedra of a cell cube around its main diagonal, one per order of
# the axes (z, y, x): corners reached by adding the axes' unit steps in turn
_KUHN = []
for _perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
    _c = [0, 0, 0]
    _tet = [tuple(_c)]
    for _a in _perm:
        _c[_a] = 1
        _tet.append(tuple(_c))
    _KUHN.append(_tet)


def _edge_point(pu, pv, fu, fv):
    """The zero of the linear interpolant between (pu, fu) and (pv, fv)."""
    t = fu / (fu - fv)
    return pu + t[:, None] * (pv - pu)


def gb_triangles(phi: np.ndarray, idf: np.ndarray):
    """The zero level {phi = 0} of a grain's box function as triangles (box-local
    coordinates (z, y, x)), by marching tetrahedra: every cell cube split into
    the six tetrahedra around its main diagonal, the level linearly
    interpolated on the edges between corners of opposite sign (phi > 0 inside
    the grain).  Each triangle carries the grain across it: the ID-field value
    most frequent among its tetrahedron's corners with phi <= 0 (the lowest id
    on ties; -1 without any).  Returns (triangles (T, 3, 3), grain (T,))."""
    nz, ny, nx = phi.shape
    if min(nz, ny, nx) < 2:
        return np.zeros((0, 3, 3)), np.zeros(0, dtype=np.int64)
    base = np.stack(np.meshgrid(np.arange(nz - 1), np.arange(ny - 1), np.arange(nx - 1), indexing="ij"),
                    axis=-1).reshape(-1, 3).astype(np.float64)
    F, P, I = [], [], []
    for tet in _KUHN:
        F.append(np.stack([phi[c[0]:nz - 1 + c[0], c[1]:ny - 1 + c[1], c[2]:nx - 1 + c[2]].ravel() for c in tet], 1))
        I.append(np.stack([idf[c[0]:nz - 1 + c[0], c[1]:ny - 1 + c[1], c[2]:nx - 1 + c[2]].ravel() for c in tet], 1))
        P.append(np.stack([base + np.array(c, dtype=np.float64) for c in tet], 1))
    F, P, I = np.concatenate(F), np.concatenate(P), np.concatenate(I)
    pos = F > 0
    npos = pos.sum(1)
    tris, grains = [], []

    def label(rows):
        out = np.full(len(rows), -1, dtype=np.int64)
        for k, r in enumerate(rows):
            ids = I[r][~pos[r]]
            ids = ids[ids >= 0]
            if ids.size:
                vals, counts = np.unique(ids, return_counts=True)
                out[k] = vals[np.argmax(counts)]            # unique sorts: ties go to the lowest id
        return out

    for n in (1, 3):                                          # one corner apart: one triangle
        rows = np.nonzero(npos == n)[0]
        if rows.size == 0:
            continue
        odd = np.argmax(pos[rows] if n == 1 else ~pos[rows], axis=1)
        others = np.array([[j for j in range(4) if j != k] for k in odd])
        pk, fk = P[rows, odd], F[rows, odd]
        pts = [_edge_point(pk, P[rows, others[:, m]], fk, F[rows, others[:, m]]) for m in range(3)]
        tris.append(np.stack(pts, 1))
        grains.append(label(rows))
    rows = np.nonzero(npos == 2)[0]                           # two and two: a quad, two triangles
    if rows.size:
        order = np.argsort(~pos[rows], axis=1, kind="stable")  # the two positive corners first
        a, b, c, d = (order[:, m] for m in range(4))
        e = lambda u, v: _edge_point(P[rows, u], P[rows, v], F[rows, u], F[rows, v])
        eac, ead, ebd, ebc = e(a, c), e(a, d), e(b, d), e(b, c)
        lab = label(rows)
        tris += [np.stack([eac, ead, ebd], 1), np.stack([eac, ebd, ebc], 1)]
        grains += [lab, lab]
    if not tris:
        return np.zeros((0, 3, 3)), np.zeros(0, dtype=np.int64)
    return np.concatenate(tris), np.concatenate(grains)


def point_triangle_distance(p: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Euclidean distance from point p to each triangle: the smaller of the
    distance to its plane's foot point, where that lies inside the triangle,
    and the distances to its three edges (clamped projections)."""
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    best = np.full(len(tris), np.inf)
    for u, v in ((a, b), (b, c), (c, a)):
        e = v - u
        t = np.clip(((p - u) * e).sum(1) / np.maximum((e * e).sum(1), 1e-300), 0.0, 1.0)
        best = np.minimum(best, np.linalg.norm(p - (u + t[:, None] * e), axis=1))
    n = np.cross(b - a, c - a)
    nn = (n * n).sum(1)
    ok = nn > 1e-24
    foot = p - (((p - a) * n).sum(1) / np.where(ok, nn, 1.0))[:, None] * n
    inside = ok.copy()
    for u, v in ((a, b), (b, c), (c, a)):
        inside &= (np.cross(v - u, foot - u) * n).sum(1) >= 0.0
    dplane = np.linalg.norm(p - foot, axis=1)
    return np.where(inside, np.minimum(best, dplane), best)


def point_triangle_distances(pts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """point_triangle_distance for several points at once: row k holds the
    distances from pts[k] to every triangle, by the same operations in the
    same order."""
    p = pts[:, None, :]
    a, b, c = tris[None, :, 0], tris[None, :, 1], tris[None, :, 2]
    best = np.full((len(pts), len(tris)), np.inf)
    for u, v in ((a, b), (b, c), (c, a)):
        e = v - u
        t = np.clip(((p - u) * e).sum(2) / np.maximum((e * e).sum(2), 1e-300), 0.0, 1.0)
        best = np.minimum(best, np.linalg.norm(p - (u + t[:, :, None] * e), axis=2))
    n = np.cross(b - a, c - a)
    nn = (n * n).sum(2)
    ok = nn > 1e-24
    foot = p - (((p - a) * n).sum(2) / np.where(ok, nn, 1.0))[:, :, None] * n
    inside = np.broadcast_to(ok, best.shape).copy()
    for u, v in ((a, b), (b, c), (c, a)):
        inside &= (np.cross(v - u, foot - u) * n).sum(2) >= 0.0
    dplane = np.linalg.norm(p - foot, axis=2)
    return np.where(inside, np.minimum(best, dplane), best)


def closest_gb_grains(phi: np.ndarray, idf: np.ndarray, tube: float, block: int = 128) -> np.ndarray:
    """The anisotropy map (R15): every cell of the box within `tube` of the
    zero level (|phi| < tube) adopts the grain across the closest triangle of
    the grain boundary (Sec. 2.1.4: each grid point takes the energy and
    mobility of the closest GB point); the other cells keep their ID-field.
    The result replaces the per-cell ID-field of R3 in Eq. (10)'s weights.
    Cells are taken `block` at a time; each takes its first closest triangle,
    as closest_gb_grain_at does."""
    tris, grains = gb_triangles(phi, idf)
    out = idf.astype(np.int64).copy()
    if len(tris) == 0:
        return out
    cells = np.argwhere(np.abs(phi) < tube)
    for k in range(0, len(cells), block):
        blk = cells[k:k + block]
        d = point_triangle_distances(blk.astype(np.float64), tris)
        out[tuple(blk.T)] = grains[np.argmin(d, axis=1)]
    return out


def closest_gb_grain_at(cell, tris: np.ndarray, grains: np.ndarray) -> int:
    """R15 for one cell (z, y, x) of a box with at least one triangle: the
    grain of the Euclidean-closest triangle (the first one on exact ties)."""
    d = point_triangle_distance(np.asarray(cell, dtype=np.float64), tris)
    return int(grains[int(np.argmin(d))])
