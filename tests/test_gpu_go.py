"""The gradient-optimisation update on the device (Sec. III) against the
oracle: the update bit for bit (the keyed draws are integer hashes, and
A - (p dt) sign is evaluated in the same order on both sides), then the
refreshed context against a fresh context built on the updated tensors."""
import numpy as np
import pytest

from oracle import peps_oracle as O
from paper_1611_09467_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_09467_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.mark.parametrize("Ly,Lx,D,Dc,prec", [(4, 4, 2, 4, "fp64"), (5, 4, 3, 6, "fp32"),
                                             (6, 6, 8, 16, "mixed_tf32")])
def test_go_step_matches_oracle_and_refreshes_the_context(Ly, Lx, D, Dc, prec):
    from paper_1611_09467_gb300.peps import PEPS
    N = Ly * Lx
    A = inputs.make_tensors(Ly, Lx, D, seed=141)
    rng = np.random.default_rng(142)
    g = rng.standard_normal(A.shape) * inputs.edge_mask(Ly, Lx, D)
    g[N // 2, 1] = 0.0                       # a block that no sample selected
    g = g.reshape(N, 2, -1)
    p = PEPS(A, Lx, Ly, D, Dc, J1=1.0, J2=0.5, prec=prec)
    A1 = p.go_step(torch.from_numpy(g).cuda(), 0.004, seed=9, step=3)
    ref = O.go_step(A, g, 0.004, 9, 3)
    assert np.array_equal(A1, ref)
    assert not np.array_equal(A1, A)
    spins = inputs.random_sz0(8, N, 143)
    S = torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).cuda()
    r1 = p.evaluate(S, logabs=True, eloc=True)
    q = PEPS(A1, Lx, Ly, D, Dc, J1=1.0, J2=0.5, prec=prec)
    r2 = q.evaluate(S, logabs=True, eloc=True)
    torch.cuda.synchronize()
    for k in ("logabs", "sign", "eloc", "status"):
        assert torch.equal(r1[k], r2[k]), k
    p.close()
    q.close()


def test_go_step_rejects_a_non_finite_gradient():
    """A NaN or infinite derivative has no sign (Sec. III moves each entry
    against the sign of its derivative): the step is refused with EINVAL and
    the context keeps its tensors."""
    from paper_1611_09467_gb300.peps import PEPS, PepsError
    Ly = Lx = 4
    D, Dc = 2, 4
    N = Ly * Lx
    A = inputs.make_tensors(Ly, Lx, D, seed=151)
    p = PEPS(A, Lx, Ly, D, Dc, J1=1.0, J2=0.5, prec="fp32")
    spins = inputs.random_sz0(8, N, 152)
    S = torch.from_numpy(inputs.pack_spins(spins).view(np.int64)).cuda()
    before = p.evaluate(S, logabs=True, eloc=True)
    g = np.random.default_rng(153).standard_normal((N, 2, D ** 4))
    for bad in (np.nan, np.inf):
        gb = g.copy()
        gb[3, 0, 5] = bad
        with pytest.raises(PepsError, match="NaN or infinite"):
            p.go_step(torch.from_numpy(gb).cuda(), 0.004, seed=1, step=0)
    after = p.evaluate(S, logabs=True, eloc=True)
    torch.cuda.synchronize()
    for k in ("logabs", "sign", "eloc"):
        assert torch.equal(before[k], after[k]), k
    # the in-place step without the host copy leaves the same context as with it
    q = PEPS(A, Lx, Ly, D, Dc, J1=1.0, J2=0.5, prec="fp32")
    mask = np.broadcast_to(inputs.edge_mask(Ly, Lx, D), (N, 2, D, D, D, D)).reshape(N, 2, -1)
    gd = torch.from_numpy(np.ascontiguousarray(g * mask)).cuda()
    p.go_step(gd, 0.004, seed=1, step=0, copy_back=False)
    A1 = q.go_step(gd, 0.004, seed=1, step=0)
    assert np.array_equal(A1, O.go_step(A, gd.cpu().numpy(), 0.004, 1, 0))
    r1, r2 = p.evaluate(S), q.evaluate(S)
    torch.cuda.synchronize()
    for k in ("logabs", "sign", "eloc"):
        assert torch.equal(r1[k], r2[k]), k
    p.close()
    q.close()


def _exact_energy_per_site(A, L, J2):
    H, basis = O.hamiltonian_sz0(L, L, 1.0, J2)
    _, psi = O.exact_sz0_wavefunction(A, L, L)
    return float(psi @ (H @ psi) / (psi @ psi)) / (L * L)


def test_go_loop_on_the_device_descends_and_respects_ed():
    """The optimisation loop of Sec. III entirely on the device, 4x4, J2 = 0,
    D = 2 (Dc = 4 is exact here), from a random start: Metropolis samples
    (peps_mc_sweep, 1024 chains) -> energy and gradient (peps_gradient) ->
    A <- A - p dt sign(dE/dA) (peps_go_step), 40 steps at dt = 0.005 (the
    paper's first step length).  The exact energy of the tensors, from the
    full S^z = 0 wavefunction, falls by more than 0.15 per site and stays
    above the ED ground energy (variational bound); the sampled energy trends
    down as well.  (The oracle's exact-gradient run from this start reaches
    -0.489 per site after 50 steps at this step length.)"""
    from paper_1611_09467_gb300.peps import PEPS
    L, D, Dc, J2 = 4, 2, 4, 0.0
    N = L * L
    A0 = inputs.make_tensors(L, L, D, seed=201)
    e_ed = O.ground_energy(L, L, 1.0, J2) / N
    p = PEPS(A0, L, L, D, Dc, J1=1.0, J2=J2, prec="fp64")
    nch = 1024
    S = torch.from_numpy(inputs.pack_spins(inputs.random_sz0(nch, N, 202)).view(np.int64)).cuda()
    p.mc_sweep(S, nsweeps=5, seed=203, chain0=0, sweep0=0)
    sampled = []
    for step in range(40):
        p.mc_sweep(S, nsweeps=2, seed=203, chain0=0, sweep0=5 + 2 * step)
        g = p.gradient(S)
        assert g["n_used"] == nch
        sampled.append(g["energy_per_site"])
        p.go_step(g["grad"], 0.005, seed=204, step=step, copy_back=(step == 39))
    A1 = p.A
    e0, e1 = _exact_energy_per_site(A0, L, J2), _exact_energy_per_site(A1, L, J2)
    print("exact energy per site: start %.5f, after 40 steps %.5f, ED %.5f" % (e0, e1, e_ed))
    print("sampled:", " ".join("%.4f" % e for e in sampled))
    assert e1 < e0 - 0.15
    assert e1 > e_ed
    assert np.mean(sampled[-5:]) < np.mean(sampled[:5]) - 0.1
    p.close()


def test_simple_update_then_go_on_the_device():
    """The paper's optimisation pipeline (Sec. III) on the device, 4x4, J2 = 0,
    D = 2: the simple update from the seeded random tensors to convergence
    (dtau = 0.01, then 0.001, each until the relative change is below 1e-6;
    peps_su_*), its PEPS as the start of the GO loop (Metropolis with 1024
    chains -> peps_gradient -> peps_go_step, 60 steps of the paper's dt
    schedule).  The exact energy of the SU state equals the oracle's SU
    energy (-0.55355), the GO steps lower it by more than 0.005 per site, and
    it stays above ED (Table I: SU -0.54557 and GO -0.570872 at D = 2)."""
    from paper_1611_09467_gb300.peps import PEPS, SimpleUpdate
    from oracle import simple_update as SU
    L, D, Dc = 4, 2, 4
    N = L * L
    Gam, lam = SU.init_state(L, L, D, 301)
    h, v = O.nn_bonds(L, L)
    su = SimpleUpdate(Gam, np.stack([lam[b] for b in h + v]), L, L, D, J1=1.0, J2=0.0)
    for dtau in (0.01, 0.001):
        for _ in range(200):
            if su.evolve(dtau, 50) < 1e-6:
                break
    A0 = su.to_peps().cpu().numpy().reshape(N, 2, D, D, D, D)
    su.close()
    e_su = _exact_energy_per_site(A0, L, 0.0)
    e_ed = O.ground_energy(L, L, 1.0, 0.0) / N
    p = PEPS(A0, L, L, D, Dc, J1=1.0, J2=0.0, prec="fp64")
    S = torch.from_numpy(inputs.pack_spins(inputs.random_sz0(1024, N, 305)).view(np.int64)).cuda()
    p.mc_sweep(S, nsweeps=5, seed=306, chain0=0, sweep0=0)
    for step in range(60):
        p.mc_sweep(S, nsweeps=2, seed=306, chain0=0, sweep0=5 + 2 * step)
        g = p.gradient(S)
        p.go_step(g["grad"], O.go_dt(step), seed=307, step=step, copy_back=(step == 59))
    e_go = _exact_energy_per_site(p.A, L, 0.0)
    print("exact energy per site: SU %.6f, after 60 GO steps %.6f, ED %.6f" % (e_su, e_go, e_ed))
    assert abs(e_su - (-0.5535529)) < 1e-5
    assert e_go < e_su - 0.005
    assert e_go > e_ed
    p.close()
