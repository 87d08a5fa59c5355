"""Pins for the FP64 oracle against facts the paper and mathematics fix.

None of these re-types the oracle's own loops.  Each reaches the same quantity
by a different route, so that a plausible slip in the oracle (a dropped
multinomial weight, a wrong image shift, a transposed contraction, a sign in
the reverse pass, the wrong element's network) fails at least one of them:

* dimer closed form: for two atoms the multinomial sum of Eq. 1 collapses to
  ``d^(2l) * (sum_m c_m phi_m W_lmk)^2`` (multinomial theorem);
* pair-dot identity: sum_a w_a (sum_j u_j A_a(r_j))^2 = sum_jj' u_j u_j' (r_j . r_j')^l,
  so rho^0 of a whole box is recomputed from dot products of neighbour vectors;
* central finite differences of the oracle energy against its reverse pass
  (Eqs. 3-5), in the positions (forces) and in a homogeneous strain (virial);
* invariances (translation, rotation of positions and cell, permutation),
  sum F = 0, extensivity of a periodic supercell;
* isolated atoms and the receptive field T * r_c of Sec. 2.2 / Fig. 2;
* neighbour counts: perfect-fcc coordination shells (crystallography, golden
  file) and self-images in a tiny cubic cell by integer enumeration.
"""

from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from synth import fcc_box, make_model, param_layout, supercell, water_box
from synth.structures import Structure

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _blocks(m):
    lay = param_layout(m.n_elem, m.T, m.n_phi, m.l_max, m.n_orb, m.h1, m.h2, m.pairs)
    p = m.params.astype(np.float64)

    def get(key):
        o, shape = lay[key]
        return p[o : o + int(np.prod(shape))].reshape(shape)

    return get


def _phi(m, d):
    """phi_m(d) for the reading: Gaussian centres linspace(0, r_c, N_phi), cosine^2 cutoff."""
    mu = np.linspace(0.0, m.r_c, m.n_phi)
    fc = np.where(d < m.r_c, (0.5 * np.cos(np.pi * d / m.r_c) + 0.5) ** 2, 0.0)
    return np.exp(-m.alpha * (d - mu) ** 2) * fc


def _mlp(get, t, e, x):
    h = x @ get((t, e, "W1")) + get((t, e, "b1"))
    h = h / (1 + np.exp(-h))
    h = h @ get((t, e, "W2")) + get((t, e, "b2"))
    h = h / (1 + np.exp(-h))
    return h @ get((t, e, "W3")) + get((t, e, "b3"))


# ------------------------------------------------------------------ Eq. 1 ---


@pytest.mark.parametrize("T", [1, 2, 3])
def test_dimer_closed_form(T):
    """Two atoms of different elements: every layer and E by the multinomial theorem."""
    m = make_model(T=T, seed=7)
    get = _blocks(m)
    rng = np.random.default_rng(3)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    d = 2.3
    pos = np.array([[0.1, -0.2, 0.3], [0.1, -0.2, 0.3] + d * u])
    species = np.array([1, 0], np.int32)  # O, H
    out = oracle.energy_forces(m, pos, species, None, want_layers=True)
    phi = _phi(m, np.array(d))
    W = get("W")
    c = get("c0")[species].copy()  # c^0 by element
    eps = np.zeros(2)
    for t in range(T):
        rho = np.zeros((2, m.n_feat))
        for i, j in ((0, 1), (1, 0)):
            for l in range(m.l_max + 1):
                s = (c[j] * phi) @ W[t, l]  # sum_m c_jm phi_m W_lmk
                rho[i, l * m.n_orb : (l + 1) * m.n_orb] = d ** (2 * l) * s**2
        np.testing.assert_allclose(out["rho"][t], rho, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(out["coef"][t], c, rtol=1e-12, atol=1e-14)
        if t < T - 1:
            c = np.stack([_mlp(get, t, species[i], rho[i]) for i in range(2)])
        else:
            eps = np.array([_mlp(get, t, species[i], rho[i])[0] for i in range(2)])
    np.testing.assert_allclose(out["atom_energy"], eps, rtol=1e-12, atol=1e-14)
    assert out["energy"] == pytest.approx(eps.sum(), rel=1e-12, abs=1e-14)


def _images(s: Structure, r_cut: float, nmax: int = 2):
    """All (i, j, r_ij) with |r_ij| < r_cut by explicit enumeration (numpy)."""
    n = s.n_atoms
    shifts = np.stack(np.meshgrid(*[np.arange(-nmax, nmax + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    out = []
    for i in range(n):
        r = s.pos[None, :, :] + (shifts @ s.cell)[:, None, :] - s.pos[i]
        d = np.linalg.norm(r, axis=-1)
        ok = d < r_cut
        ok[np.all(shifts == 0, axis=1), i] = False
        si, j = np.nonzero(ok)
        out.append((i, j, r[si, j]))
    return out


def test_rho0_pair_dot_identity():
    """rho^0 of a water box via sum_jj' u_j u_j' (r_ij . r_ij')^l (no monomials)."""
    m = make_model(T=1, seed=11)
    get = _blocks(m)
    s = water_box(16, seed=5)  # 48 atoms, L = 7.82 A < 2 r_c: several images per pair
    out = oracle.energy_forces(m, s.pos, s.species, s.cell, want_layers=True)
    W = get("W")[0]
    c0 = get("c0")
    for i, j, r in _images(s, m.r_c):
        d = np.linalg.norm(r, axis=1)
        phi = np.stack([_phi(m, x) for x in d]) if len(d) else np.zeros((0, m.n_phi))
        dots = r @ r.T
        for l in range(m.l_max + 1):
            u = (c0[s.species[j]] * phi) @ W[l]  # (n_nb, n_orb)
            rho = np.einsum("ak,bk,ab->k", u, u, dots**l)
            np.testing.assert_allclose(out["rho"][0][i, l * m.n_orb : (l + 1) * m.n_orb], rho, rtol=1e-10, atol=1e-12)


def test_rho0_pair_products_bilinear_identity():
    """The orbital-pair features: rho_(l,(k,k')) = sum_a w_a g_ak g_ak' equals
    sum_jj' u_jk u_j'k' (r_ij . r_ij')^l (bilinear form of the multinomial
    theorem), and its diagonal equals Eq. 1's squares of the same orbitals."""
    m = make_model(T=1, seed=11, pairs=True)
    get = _blocks(m)
    s = water_box(16, seed=5)
    out = oracle.energy_forces(m, s.pos, s.species, s.cell, want_layers=True)
    W = get("W")[0]
    c0 = get("c0")
    K = m.n_orb
    iu = np.triu_indices(K)
    per_l = K * (K + 1) // 2
    for i, j, r in _images(s, m.r_c):
        d = np.linalg.norm(r, axis=1)
        phi = np.stack([_phi(m, x) for x in d]) if len(d) else np.zeros((0, m.n_phi))
        dots = r @ r.T
        for l in range(m.l_max + 1):
            u = (c0[s.species[j]] * phi) @ W[l]
            rho = np.einsum("ak,bq,ab->kq", u, u, dots**l)[iu]
            np.testing.assert_allclose(out["rho"][0][i, l * per_l : (l + 1) * per_l], rho, rtol=1e-10, atol=1e-12)
    # the diagonal pairs are the squares model's features (same c0 and W: same seed and n_orb)
    sq = make_model(T=1, seed=11, n_orb=K)
    out_sq = oracle.energy_forces(sq, s.pos, s.species, s.cell, want_layers=True)
    diag = [q for q, (a, b) in enumerate(zip(*iu)) if a == b]
    for l in range(m.l_max + 1):
        np.testing.assert_allclose(out["rho"][0][:, l * per_l + np.array(diag)], out_sq["rho"][0][:, l * K : (l + 1) * K],
                                   rtol=1e-12, atol=1e-14)


# -------------------------------------------------------------- Eqs. 3-5 ----


@pytest.mark.parametrize("pairs", [False, True], ids=["squares", "pairs"])
@pytest.mark.parametrize(
    "make",
    [lambda: water_box(8, seed=2), lambda: fcc_box(2, seed=4, sigma=0.1)],
    ids=["water24", "fcc32"],
)
def test_forces_match_central_differences(make, pairs):
    s = make()
    m = make_model(T=3, seed=5, pairs=pairs)
    out = oracle.energy_forces(m, s.pos, s.species, s.cell)
    h = 1e-5
    fd = np.zeros_like(s.pos)
    for a in range(s.n_atoms):
        for k in range(3):
            p = s.pos.copy()
            p[a, k] += h
            ep = oracle.energy_forces(m, p, s.species, s.cell)["energy"]
            p[a, k] -= 2 * h
            em = oracle.energy_forces(m, p, s.species, s.cell)["energy"]
            fd[a, k] = -(ep - em) / (2 * h)
    assert np.abs(out["forces"]).max() > 1e-4  # the test is not vacuous (1e3 x the bar)
    np.testing.assert_allclose(out["forces"], fd, atol=1e-7, rtol=0)


@pytest.mark.parametrize(
    "make",
    [lambda: water_box(8, seed=2), lambda: fcc_box(2, seed=4, sigma=0.1)],
    ids=["water24", "fcc32"],
)
def test_virial_is_minus_strain_derivative(make):
    """W_ab = -dE/d eps_ab: central differences of E under the homogeneous strain
    x -> (I + eps) x applied to every position and every lattice vector; W is
    symmetric because E is invariant under rotations."""
    s = make()
    m = make_model(T=3, seed=5)
    out = oracle.energy_forces(m, s.pos, s.species, s.cell)
    h = 1e-5
    fd = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            e = np.zeros((3, 3))
            e[a, b] = h
            # row vectors: x' = x (I + eps)^T
            ep = oracle.energy_forces(m, s.pos @ (np.eye(3) + e).T, s.species, s.cell @ (np.eye(3) + e).T)["energy"]
            em = oracle.energy_forces(m, s.pos @ (np.eye(3) - e).T, s.species, s.cell @ (np.eye(3) - e).T)["energy"]
            fd[a, b] = -(ep - em) / (2 * h)
    assert np.abs(out["virial"]).max() > 1e-3  # not vacuous
    np.testing.assert_allclose(out["virial"], fd, atol=1e-6, rtol=0)
    np.testing.assert_allclose(out["virial"], out["virial"].T, atol=1e-9, rtol=0)


# ------------------------------------------------------------ invariances ---


def test_invariances_and_extensivity():
    m = make_model(T=3)
    s = water_box(16, seed=9)
    base = oracle.energy_forces(m, s.pos, s.species, s.cell)
    E, F = base["energy"], base["forces"]
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-10)
    # translation
    t = oracle.energy_forces(m, s.pos + np.array([3.3, -11.7, 0.45]), s.species, s.cell)
    assert t["energy"] == pytest.approx(E, rel=1e-11, abs=1e-11)
    np.testing.assert_allclose(t["forces"], F, atol=1e-9)
    # rotation of positions and cell together
    rng = np.random.default_rng(0)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    r = oracle.energy_forces(m, s.pos @ q.T, s.species, s.cell @ q.T)
    assert r["energy"] == pytest.approx(E, rel=1e-11, abs=1e-11)
    np.testing.assert_allclose(r["forces"], F @ q.T, atol=1e-9)
    # permutation
    perm = rng.permutation(s.n_atoms)
    p = oracle.energy_forces(m, s.pos[perm], s.species[perm], s.cell)
    assert p["energy"] == pytest.approx(E, rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(p["forces"], F[perm], atol=1e-10)
    np.testing.assert_allclose(p["atom_energy"], base["atom_energy"][perm], atol=1e-12)
    # extensivity: a 2x1x2 periodic supercell carries 4 copies of every atom energy
    big = supercell(s, (2, 1, 2))
    b = oracle.energy_forces(m, big.pos, big.species, big.cell)
    assert b["energy"] == pytest.approx(4 * E, rel=1e-11)
    np.testing.assert_allclose(b["atom_energy"], np.tile(base["atom_energy"], 4), atol=1e-11)
    np.testing.assert_allclose(b["forces"], np.tile(F, (4, 1)), atol=1e-9)


def test_isolated_atoms_have_zero_energy_and_force():
    m = make_model(T=3)
    s = Structure(np.array([[1.0, 2.0, 3.0], [11.0, 2.0, 3.0]]), np.array([0, 2], np.int32), np.eye(3) * 20.0)
    out = oracle.energy_forces(m, s.pos, s.species, s.cell, want_layers=True)
    assert out["energy"] == 0.0
    assert np.all(out["forces"] == 0.0)
    assert np.all(out["rho"] == 0.0)


@pytest.mark.parametrize("T", [1, 2, 3])
def test_receptive_field_is_T_times_rc(T):
    """eps_i ignores atoms farther than T r_c (a chain of links of length < r_c)."""
    m = make_model(T=T, seed=21)
    # a linear chain with 4.0 A links: atom k sits at 4k A, so atom 0 is reached
    # after k message-passing layers through the chain.
    n = 6
    pos = np.zeros((n, 3))
    pos[:, 0] = 4.0 * np.arange(n)
    sp = np.array([1, 0, 1, 0, 1, 0], np.int32)
    base = oracle.energy_forces(m, pos, sp, None)["atom_energy"][0]
    for k in range(1, n):
        moved = pos.copy()
        moved[k, 1] += 0.3  # bend the chain at atom k
        e0 = oracle.energy_forces(m, moved, sp, None)["atom_energy"][0]
        if k > T:
            assert e0 == base, (k, T)
        else:
            assert e0 != base, (k, T)


# ---------------------------------------------------------- neighbours ------


def _golden_shells():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "fcc_shells.txt")) if ln.strip() and not ln.startswith("#")]
    return {int(a): int(b) for a, b in rows}


@pytest.mark.parametrize("r_cut,n_shells", [(5.0, 3), (6.0, 5)])
def test_perfect_fcc_coordination(r_cut, n_shells):
    a = 3.615
    s = fcc_box(4, a=a, sigma=0.0)
    shells = _golden_shells()
    expect = sum(shells[k] for k in range(1, 7) if a * math.sqrt(k / 2) < r_cut)
    assert expect == sum(shells[k] for k in range(1, n_shells + 1))
    i, j, sh = oracle.neighbors(s.pos, s.cell, r_cut)
    counts = np.bincount(i, minlength=s.n_atoms)
    assert np.all(counts == expect)


def test_self_images_tiny_cubic_cell():
    """One atom in a 2.5 A cube: neighbours are the lattice points n with 2.5|n| < 6."""
    L, r_cut = 2.5, 6.0
    r = np.arange(-3, 4)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    nn = (n * n).sum(1)
    expect = int(((nn > 0) & (L * L * nn < r_cut * r_cut)).sum())
    i, j, sh = oracle.neighbors(np.array([[0.3, 1.1, 2.4]]), np.eye(3) * L, r_cut)
    assert len(i) == expect == 56
    got = {tuple(x) for x in sh}
    assert len(got) == expect


def test_neighbor_set_triclinic_matches_enumeration():
    rng = np.random.default_rng(1)
    cell = np.array([[6.0, 0.0, 0.0], [1.7, 5.5, 0.0], [-1.1, 0.9, 6.3]])
    frac = rng.random((10, 3))
    pos = frac @ cell + rng.normal(0, 2.0, size=(10, 3))  # some atoms outside the cell
    s = Structure(pos, np.zeros(10, np.int32), cell)
    i, j, sh = oracle.neighbors(pos, cell, 4.7)
    got = {(a, b, *c) for a, b, c in zip(i.tolist(), j.tolist(), sh.tolist())}
    shifts = np.stack(np.meshgrid(*[np.arange(-5, 6)] * 3, indexing="ij"), -1).reshape(-1, 3)
    want = set()
    for a in range(10):
        r = pos[None, :, :] + (shifts @ cell)[:, None, :] - pos[a]
        d = np.linalg.norm(r, axis=-1)
        for si, b in zip(*np.nonzero(d < 4.7)):
            if b == a and np.all(shifts[si] == 0):
                continue
            want.add((a, int(b), *shifts[si].tolist()))
    assert got == want
    assert len(got) == len(i)


def test_bad_geometry_is_rejected():
    m = make_model(T=1)
    with pytest.raises(oracle.OracleError):
        oracle.energy_forces(m, np.array([[0.0, 0.0, np.nan]]), np.zeros(1, np.int32), np.eye(3) * 10)
    with pytest.raises(oracle.OracleError):
        oracle.energy_forces(m, np.zeros((2, 3)), np.zeros(2, np.int32), np.eye(3) * 10)  # coincident
    with pytest.raises(oracle.OracleError):
        oracle.energy_forces(m, np.zeros((1, 3)), np.zeros(1, np.int32), np.zeros((3, 3)))  # singular cell
    with pytest.raises(oracle.OracleError):
        oracle.energy_forces(m, np.zeros((1, 3)), np.array([7], np.int32), np.eye(3) * 10)  # species
