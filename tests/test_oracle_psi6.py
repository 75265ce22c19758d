"""Pins of the oracle's bond-orientational order (Eq. 8)."""
import numpy as np
import pytest


def _shell_system(oracle_mod, form, theta0, radii, angles=None):
    """Seven disks in a 40 x 40 box: one centre and six neighbours."""
    N, L = 7, 40.0
    o = oracle_mod.OracleChain(N, N * np.pi / L ** 2, 0.1, 1, form=form)
    Lr = o.geometry()["L"]
    c = np.array([Lr / 2, Lr / 2])
    if angles is None:
        angles = theta0 + np.arange(6) * np.pi / 3
    xy = [c] + [c + r * np.array([np.cos(a), np.sin(a)]) for r, a in zip(radii, angles)]
    xy = np.array(xy)
    o.set_positions(xy)
    return o, o.positions()


@pytest.mark.parametrize("form,tol", [("fp64", 1e-12), ("fixed", 3e-6)])
@pytest.mark.parametrize("theta0", [0.0, 0.1, 0.7, 2.0])
def test_hexagonal_shell(oracle_mod, form, tol, theta0):
    """A centre with six neighbours at angles theta0 + k pi/3 has
    psi = exp(6 i theta0) exactly."""
    radii = 2.3 * (1 + 0.01 * np.arange(6))
    o, _ = _shell_system(oracle_mod, form, theta0, radii)
    loc, _ = o.psi6()
    assert abs(loc[0] - np.exp(6j * theta0)) < tol


@pytest.mark.parametrize("form,tol", [("fp64", 1e-12), ("fixed", 3e-6)])
def test_irregular_shell_against_trig(oracle_mod, form, tol):
    """Arbitrary bond angles: psi = mean exp(6 i phi_k) with phi from atan2 on
    the global minimum-image vectors (numpy trigonometry, independent of the
    z^6 / |z|^6 algebra)."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        ang = np.sort(rng.uniform(0, 2 * np.pi, 6))
        radii = 2.2 + 0.4 * rng.uniform(size=6)
        o, xy = _shell_system(oracle_mod, form, 0.0, radii, angles=ang)
        d = xy[1:] - xy[0]
        want = np.mean(np.exp(6j * np.arctan2(d[:, 1], d[:, 0])))
        loc, _ = o.psi6()
        assert abs(loc[0] - want) < tol


def _liquid(oracle_mod, form):
    o = oracle_mod.OracleChain(256, 0.70, 0.15, 8, form=form)
    o.sweep(300)
    return o


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_covariance(oracle_mod, form):
    """Rotating the box by 90 degrees multiplies every psi_j by exp(6 i pi/2)
    = -1; reflecting x -> -x conjugates it; swapping x and y gives -conj.
    Bit-exact in the fixed form, where the integer bond vectors map exactly."""
    o = _liquid(oracle_mod, form)
    loc, glob = o.psi6()
    xy = o.positions()
    L = o.geometry()["L"]
    o2 = oracle_mod.OracleChain(256, 0.70, 0.15, 8, form=form)
    tol = 0.0 if form == "fixed" else 1e-9
    for tf, fn in [(lambda p: np.stack([(L - p[:, 1]) % L, p[:, 0]], 1), lambda z: -z),
                   (lambda p: np.stack([(L - p[:, 0]) % L, p[:, 1]], 1), np.conj),
                   (lambda p: np.stack([p[:, 1], p[:, 0]], 1), lambda z: -np.conj(z))]:
        o2.set_positions(tf(xy))
        l2, g2 = o2.psi6()
        assert np.abs(l2 - fn(loc)).max() <= tol
        assert abs(g2 - fn(glob)) <= tol + 1e-15


@pytest.mark.parametrize("form", ["fp64", "fixed"])
@pytest.mark.parametrize("eta", [0.70, 0.15])
def test_ring_search_equals_brute(oracle_mod, form, eta):
    """The expanding cell-ring search must find exactly the neighbours of a
    scan over all disks; at eta = 0.15 the sixth neighbour often lies beyond
    the first 5 x 5 cell stencil."""
    o = oracle_mod.OracleChain(256, eta, 0.15 if eta > 0.5 else 1.0, 8, form=form)
    for _ in range(4 if eta > 0.5 else 12):
        o.sweep(100)
        a, ga = o.psi6()
        b, gb = o.psi6(brute=True)
        assert np.array_equal(a, b) and ga == gb
        assert np.all(np.abs(a) <= 1 + 1e-6)


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_global_is_exactly_rounded_mean(oracle_mod, form):
    """Psi_6 = (1/N) sum_j psi_j (Eq. 8) with each part's sum rounded once:
    checked against exact rational arithmetic on a liquid state, and
    unchanged (bit for bit) when the disks are summed in another order."""
    from fractions import Fraction
    o = _liquid(oracle_mod, form)
    loc, glob = o.psi6()
    N = loc.size
    for part, got in ((loc.real, glob.real), (loc.imag, glob.imag)):
        exact = sum((Fraction(float(v)) for v in part), Fraction(0))
        assert got == float(exact) / N
    perm = np.random.default_rng(1).permutation(N)
    assert oracle_mod.psi6_mean(loc[perm]) == glob


def test_exact_mean_keeps_small_terms():
    """A running double sum drops 2^20 terms of 2^-60 added to 1; the
    exactly rounded sum keeps them: 1 + 2^-40."""
    import oracle
    z = np.array([1.0] + [2.0 ** -60] * (1 << 20)) * (1 - 1j)
    n = z.size
    got = oracle.psi6_mean(z)
    assert got == complex((1 + 2.0 ** -40) / n, -(1 + 2.0 ** -40) / n)
    naive = 0.0
    for v in z.real[:1000]:
        naive += v
    assert naive == 1.0


@pytest.mark.parametrize("form", ["fp64", "fixed"])
def test_square_lattice_ties_broken_by_id(oracle_mod, form):
    """A square lattice: four nearest neighbours at 0, 90, 180, 270 degrees
    contribute exp(6i phi) = 1, -1, 1, -1 (sum 0), and the 5th and 6th are two
    of the four diagonal neighbours, all at the same distance: the tie rule
    (smaller id first) picks the two of smallest id.  Diagonals at 45 / 225
    degrees give exp(6i phi) = -i, at 135 / 315 degrees +i; so psi_j is the
    mean of those two picks, computed here from the lattice indices alone."""
    n = 16
    N = n * n
    o = oracle_mod.OracleChain(N, 0.5, 0.1, 1, form=form)  # square start lattice, no sweep
    L = o.geometry()["L"]
    xy = o.positions()
    a = L / n
    col = np.rint(xy[:, 0] / a - 0.5).astype(int) % n
    row = np.rint(xy[:, 1] / a - 0.5).astype(int) % n
    idx = {(int(c), int(r)): i for i, (c, r) in enumerate(zip(col, row))}
    loc, _ = o.psi6()
    for i in range(N):
        c, r = int(col[i]), int(row[i])
        diag = [(idx[((c + dx) % n, (r + dy) % n)], dx, dy) for dx in (-1, 1) for dy in (-1, 1)]
        diag.sort()
        val = sum((-1j if dx * dy > 0 else 1j) for _, dx, dy in diag[:2]) / 6
        assert abs(loc[i] - val) < (1e-12 if form == "fp64" else 1e-6), (i, loc[i], val)
