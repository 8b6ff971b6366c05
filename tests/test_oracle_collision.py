"""Single-site pins of the oracle's collision operator (Sec. II A-B) against
closed forms and exact invariants. CPU only."""
import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0


def _lattice(vs, **params):
    shape = (1, 1, 1) if vs == O.D2Q9 else (1, 1, 1)
    p = dict(velset=vs, tau_amb=0.9, A=0.05, beta=0.7)
    p.update(params)
    return O.Oracle(shape, params=p, geom=dict(nozzle=0, z_mode=O.Z_PERIODIC),
                    rheo=dict(law=O.NEWTONIAN, nu0=(1.1 - 0.5) / 3, tau_min=0.501, tau_max=5.0))


def _feq(c, w, rho, u):
    cu = c @ u
    return rho * w * (1 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - (u @ u) / (2 * CS2))


def _state(vs, rng, rhoY=0.55, rhoB=0.45, u=None, neq=1e-3, grad=None):
    """Populations near equilibrium, and neighbour densities with a linear
    phase field rhoN(x + c_i) = a + grad . c_i and total density 1."""
    c, w, B = O.velset(vs)
    Q = len(w)
    if u is None:
        u = np.array([0.01, -0.02, 0.015]) if vs == O.D3Q19 else np.array([0.01, 0.0, 0.015])
    fin = np.stack([_feq(c, w, rhoY, u), _feq(c, w, rhoB, u)])
    if neq:
        pert = rng.normal(size=(2, Q)) * neq
        pert -= pert.mean(axis=1, keepdims=True)  # keeps component masses
        fin = fin + pert * w
    if grad is None:
        grad = np.array([0.03, 0.02, -0.04]) if vs == O.D3Q19 else np.array([0.03, 0.0, -0.04])
    a = (rhoY - rhoB) / (rhoY + rhoB)
    rn = a + c @ grad
    nbr = np.stack([(1 + rn) / 2, (1 - rn) / 2])
    return c, w, B, fin, nbr, np.asarray(grad, float)


@pytest.mark.parametrize("vs", [O.D2Q9, O.D3Q19])
def test_component_mass_and_total_momentum_conserved(vs):
    rng = np.random.default_rng(1)
    L = _lattice(vs)
    c, w, B, fin, nbr, g = _state(vs, rng)
    out, aux = L.collide_one(fin, nbr)
    for k in range(2):
        assert out[k].sum() == pytest.approx(fin[k].sum(), abs=1e-15)
    mom_in = (fin.sum(0)[:, None] * c).sum(0)
    mom_out = (out.sum(0)[:, None] * c).sum(0)
    assert np.allclose(mom_out, mom_in, rtol=0, atol=2e-15)


@pytest.mark.parametrize("vs", [O.D2Q9, O.D3Q19])
def test_isotropic_gradient_exact_for_linear_field(vs):
    """Eq. 12 is exact for a linear field: |grad rhoN| = |b|."""
    rng = np.random.default_rng(2)
    L = _lattice(vs)
    c, w, B, fin, nbr, g = _state(vs, rng)
    out, aux = L.collide_one(fin, nbr)
    assert aux[1] == pytest.approx(np.linalg.norm(g), rel=1e-14)


@pytest.mark.parametrize("vs", [O.D2Q9, O.D3Q19])
def test_perturbation_stress_closed_form(vs):
    """With populations at equilibrium at rest (BGK leaves them unchanged) and no
    recolouring, the total post-collision second moment differs from the
    equilibrium one by exactly (A/9)|grad rhoN|(n n - I) (Eq. 10 with the
    lattice identities), applied once to the mixture; mass and momentum of the
    perturbation vanish."""
    rng = np.random.default_rng(3)
    A = 0.07
    L = _lattice(vs, A=A, beta=0.0)
    c, w, B, fin, nbr, g = _state(vs, rng, u=np.zeros(3), neq=0.0)
    out, aux = L.collide_one(fin, nbr)
    dtot = out.sum(0) - fin.sum(0)
    n = g / np.linalg.norm(g)
    axes = [0, 2] if vs == O.D2Q9 else [0, 1, 2]
    M = np.einsum("i,ia,ib->ab", dtot, c, c)
    for a in axes:
        for b in axes:
            expect = A / 9 * np.linalg.norm(g) * (n[a] * n[b] - (a == b))
            assert M[a, b] == pytest.approx(expect, abs=2e-15)
    assert abs(dtot.sum()) < 2e-15
    assert np.allclose((dtot[:, None] * c).sum(0), 0.0, rtol=0, atol=2e-15)


@pytest.mark.parametrize("vs", [O.D2Q9, O.D3Q19])
@pytest.mark.parametrize("gscale", [1.0, 1e-3, 1e-9])
def test_recolouring_closed_form(vs, gscale):
    """Recolouring (Eq. 14-16) leaves the total f* unchanged and moves ink
    momentum along +grad rhoN by exactly beta (rhoY rhoB / rho) kappa n, with
    kappa = sum_i w_i c_ix^2/|c_i| (phi = w at density ratio one) and
    n = grad rhoN / |grad rhoN|: cos(phi_i) of Eq. 16 as printed, at full size
    for any gradient above the rounding floor (here down to 1e-9 of the
    interface scale)."""
    rng = np.random.default_rng(4)
    beta = 0.6
    L0 = _lattice(vs, beta=0.0)
    L1 = _lattice(vs, beta=beta)
    g0 = np.array([0.03, 0.02, -0.04]) if vs == O.D3Q19 else np.array([0.03, 0.0, -0.04])
    c, w, B, fin, nbr, g = _state(vs, rng, grad=g0 * gscale)
    o0, _ = L0.collide_one(fin, nbr)
    o1, _ = L1.collide_one(fin, nbr)
    assert np.allclose(o1.sum(0), o0.sum(0), rtol=0, atol=2e-15)
    rY, rB = fin[0].sum(), fin[1].sum()
    rho = rY + rB
    cn = np.sqrt((c * c).sum(1))
    kappa = sum(w[i] * c[i, 0] ** 2 / cn[i] for i in range(1, len(w)))
    assert kappa == pytest.approx((1 + np.sqrt(2)) / 9 if vs == O.D3Q19 else (4 + np.sqrt(2)) / 18, rel=1e-15)
    n = g / np.linalg.norm(g)
    shift = ((o1[0] - o0[0])[:, None] * c).sum(0)
    # the neighbour densities carry the gradient to ~1e-16 absolute, so its
    # direction is known to ~1e-16 / |grad|
    tol = 2e-15 + 4e-16 / (np.linalg.norm(g) / 0.054)
    assert np.allclose(shift, beta * rY * rB / rho * kappa * n, rtol=0, atol=tol)
    # and each direction's recolouring term is beta rhoY rhoB/rho^2 cos(phi_i) rho w_i
    cosp = np.zeros(len(w))
    cosp[1:] = (c[1:] @ g) / (cn[1:] * np.linalg.norm(g))
    assert np.allclose(o1[0] - o0[0], beta * rY * rB / rho ** 2 * cosp * rho * w, rtol=0, atol=tol)


@pytest.mark.parametrize("vs", [O.D2Q9, O.D3Q19])
def test_uniform_equilibrium_is_fixed_point(vs):
    """A uniform two-component state at equilibrium with any velocity is left
    unchanged (no gradient, no non-equilibrium stress)."""
    rng = np.random.default_rng(5)
    L = _lattice(vs)
    c, w, B, fin, nbr, g = _state(vs, rng, neq=0.0, grad=np.zeros(3))
    out, aux = L.collide_one(fin, nbr)
    assert np.allclose(out, fin, rtol=0, atol=2e-15)


def test_exact_difference_forcing():
    """Body force by the exact difference method (Eq. 29 is added the same way):
    the momentum changes by exactly F = rho g per step, component masses are
    untouched, and the reported velocity is u + F/(2 rho)."""
    rng = np.random.default_rng(6)
    gvec = np.array([1e-4, -2e-4, 3e-5])
    L = _lattice(O.D3Q19, body_force=tuple(gvec))
    c, w, B, fin, nbr, g = _state(O.D3Q19, rng)
    out, aux = L.collide_one(fin, nbr)
    rho = fin.sum()
    dm = (out.sum(0)[:, None] * c).sum(0) - (fin.sum(0)[:, None] * c).sum(0)
    assert np.allclose(dm, rho * gvec, rtol=0, atol=2e-15)
    u = (fin.sum(0)[:, None] * c).sum(0) / rho
    assert np.allclose(aux[2:5], u + gvec / 2, rtol=0, atol=2e-15)
    for k in range(2):
        assert out[k].sum() == pytest.approx(fin[k].sum(), abs=1e-15)


def test_drag_only_near_substrate():
    """Drag F = -gamma rho_Y u (Eq. 29) acts within drag_height of the substrate."""
    rng = np.random.default_rng(7)
    gam = 0.05
    L = _lattice(O.D3Q19, drag_gamma=gam, drag_height=4.0)
    c, w, B, fin, nbr, g = _state(O.D3Q19, rng)
    rho = fin.sum()
    rY = fin[0].sum()
    u = (fin.sum(0)[:, None] * c).sum(0) / rho
    out_in, _ = L.collide_one(fin, nbr, z_wall_dist=3.5)
    out_out, _ = L.collide_one(fin, nbr, z_wall_dist=4.5)
    dm_in = (out_in.sum(0)[:, None] * c).sum(0) - (fin.sum(0)[:, None] * c).sum(0)
    dm_out = (out_out.sum(0)[:, None] * c).sum(0) - (fin.sum(0)[:, None] * c).sum(0)
    assert np.allclose(dm_in, -gam * rY * u, rtol=0, atol=2e-15)
    assert np.allclose(dm_out, 0.0, rtol=0, atol=2e-15)


def test_colour_swap_symmetry_single_site():
    rng = np.random.default_rng(8)
    L = O.Oracle((1, 1, 1), params=dict(tau_amb=0.8, A=0.05, beta=0.7),
                 geom=dict(nozzle=0, z_mode=O.Z_PERIODIC),
                 rheo=dict(law=O.NEWTONIAN, nu0=(0.8 - 0.5) / 3, tau_min=0.501, tau_max=5.0))
    c, w, B, fin, nbr, g = _state(O.D3Q19, rng)
    out, _ = L.collide_one(fin, nbr)
    outs, _ = L.collide_one(fin[::-1].copy(), nbr[::-1].copy())
    assert np.allclose(outs[::-1], out, rtol=0, atol=2e-15)


# --------------------------------------------------------------------------
# local relaxation time (Eq. 17, 23-25)
# --------------------------------------------------------------------------

def test_power_law_root_closed_form_n_half():
    """For n = 1/2, gdot tau(gdot) = s reads gdot/2 + 3 K sqrt(gdot) = s, whose
    root is sqrt(gdot) = -3K + sqrt(9K^2 + 2s)."""
    K = 0.02
    rheo = dict(law=O.POWER_LAW, n=0.5, K=K, tau_min=0.5001, tau_max=1e6)
    for S, rY in [(1e-4, 1.0), (3e-3, 0.8), (0.05, 1.2)]:
        s = S / (rY * CS2)
        q = -3 * K + np.sqrt(9 * K * K + 2 * s)
        tau, gd = O.solve_tau_ink(rheo, S, rY)
        assert gd == pytest.approx(q * q, rel=1e-13)
        assert tau == pytest.approx(0.5 + 3 * K / q, rel=1e-13)


def test_root_satisfies_eq24_and_clamps():
    rheo = dict(law=O.POWER_LAW, n=0.6, K=0.05, tau_min=0.51, tau_max=2.0)
    # middle branch
    S, rY = 2e-2, 1.0
    tau, gd = O.solve_tau_ink(rheo, S, rY)
    assert gd == pytest.approx(S / (rY * tau * CS2), rel=1e-13)
    assert 0.51 < tau < 2.0
    # tiny stress: nu -> large, clamped at tau_max, root gdot = s / tau_max
    tau, gd = O.solve_tau_ink(rheo, 1e-9, 1.0)
    assert tau == 2.0 and gd == pytest.approx(1e-9 / CS2 / 2.0, rel=1e-13)
    # huge stress: clamped at tau_min
    tau, gd = O.solve_tau_ink(rheo, 1000.0, 1.0)
    assert tau == 0.51 and gd == pytest.approx(1000.0 / CS2 / 0.51, rel=1e-13)
    # no stress: power law at zero shear is clamped at tau_max
    tau, gd = O.solve_tau_ink(rheo, 0.0, 1.0)
    assert tau == 2.0


def test_cross_reduces_to_newtonian_and_power_law():
    # nu0 = nu_inf: Cross is Newtonian whatever the shear rate
    r = dict(law=O.CROSS, nu0=0.2, nu_inf=0.2, lam=3.0, n=0.7, tau_min=0.51, tau_max=3.0)
    for S in (1e-6, 1e-3, 0.1):
        tau, _ = O.solve_tau_ink(r, S, 1.0)
        assert tau == 0.5 + 0.2 / CS2
    # nu_inf = 0 and lambda gdot >> 1: power law with n_pl = 1 - n, K = nu0 lambda^-n
    lam, n, nu0 = 1e16, 0.4, 0.3
    rc = dict(law=O.CROSS, nu0=nu0, nu_inf=0.0, lam=lam, n=n, tau_min=0.5001, tau_max=1e9)
    rp = dict(law=O.POWER_LAW, n=1 - n, K=nu0 * lam ** (-n), tau_min=0.5001, tau_max=1e9)
    for S in (1e-4, 1e-2):
        t1, g1 = O.solve_tau_ink(rc, S, 1.0)
        t2, g2 = O.solve_tau_ink(rp, S, 1.0)
        assert (t1 - 0.5) == pytest.approx(t2 - 0.5, rel=1e-4)
        assert g1 == pytest.approx(g2, rel=1e-4)


def test_recolouring_direction_floor():
    """Eq. 16 has no value where grad rhoN = 0 (0/0). A computed gradient at or
    below the rounding level of the arithmetic (the floor, 2^8 units of
    rounding: 2^-45 for FP64, 2^-16 for a path computing in FP32) has no
    meaningful direction either: there, and only there, cos(phi_i) = 0 and the
    recolouring leaves f^Y = (rho_Y/rho) f*. Just above the floor it acts at
    full size."""
    rng = np.random.default_rng(9)
    for floor in (2.0 ** -45, 2.0 ** -16):
        L0 = _lattice(O.D3Q19, beta=0.0, grad_floor=floor)
        L1 = _lattice(O.D3Q19, beta=0.7, grad_floor=floor)
        for gmag, acts in ((0.0, False), (1e-17, False), (0.5 * floor, False), (2.0 * floor, True)):
            c, w, B, fin, nbr, g = _state(O.D3Q19, rng, grad=np.array([gmag, 0.0, 0.0]))
            o0, a0 = L0.collide_one(fin, nbr)
            o1, a1 = L1.collide_one(fin, nbr)
            d = np.abs(o1 - o0).max()
            if acts:
                # the recolouring term's size: beta rhoY rhoB / rho^2 * rho w_i
                rY, rB = fin[0].sum(), fin[1].sum()
                assert d == pytest.approx(0.7 * rY * rB / (rY + rB) / 18, rel=0.05)
            else:
                assert d == 0.0


def test_default_floor_is_fp64_rounding_level():
    assert O.grad_floor({}) == 2.0 ** -45
    assert O.grad_floor({"storage": "f32"}) == 2.0 ** -16
    assert O.grad_floor({"storage": "f16dev", "grad_floor": 1e-3}) == 1e-3


@pytest.mark.parametrize("cy", [1e-13, 1e-8])
def test_gradient_keeps_relative_precision_in_the_ink_tail(cy):
    """Far in the ambient the ink fraction is tiny and rho^N = -1 + 2 c_Y; its
    gradient (Eq. 12) must still come out with the relative precision of the
    ink densities, since the direction of Eq. 16 is read from it there. With
    c_Y(x + c_i) = cy (1 + g.c_i) the gradient is 2 cy g exactly (Eq. 12 is
    exact for linear fields), and the recolouring direction is g/|g|."""
    L = _lattice(O.D3Q19, beta=0.7)
    c, w, B = O.velset(O.D3Q19)
    g = np.array([0.3, -0.2, 0.4])
    cyn = cy * (1 + c @ g)
    nbr = np.stack([cyn, 1 - cyn])
    u = np.zeros(3)
    fin = np.stack([cy * w, (1 - cy) * w])
    out, aux = L.collide_one(fin, nbr)
    assert aux[1] == pytest.approx(2 * cy * np.linalg.norm(g), rel=1e-9)
    # the ink's recolouring momentum points along +g to the same precision
    L0 = _lattice(O.D3Q19, beta=0.0)
    o0, _ = L0.collide_one(fin, nbr)
    shift = ((out[0] - o0[0])[:, None] * c).sum(0)
    n = shift / np.linalg.norm(shift)
    assert np.allclose(n, g / np.linalg.norm(g), rtol=0, atol=1e-9)
