"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: relative L2 <= 1e-4 for FP32 fields and spectra (the bar the
method's target states); FP64 tier <= 1e-11; 16-bit storage tiers are
reported with a loose bound.  Inputs are seeded; sizes span several tiles
with ragged tails; both signs of v, zero v, narrow layers (several
boundaries per lane), non-uniform mu, moving matter and piecewise-linear
profiles are covered.
"""
import numpy as np
import pytest

from helpers import make_oracle, make_sim, rel_l2
from paper_2304_06586_gb300 import binding as gb
from paper_2304_06586_gb300 import workloads as w

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
SHAPES = [(16, 16), (8, 16), (16, 24, 8), (20, 16), (20, 24), (20, 32), (24, 24)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    gb.load()


def _mixed_workload(seed=7, kind=w.PERTURBATION, interp=w.LAYERS):
    """Ragged instances: tiny, tile-boundary and multi-tile sizes, both signs of v."""
    rng = np.random.default_rng(seed)
    sizes = [1, 7, 32, 33, 100, 517, 1000, 3001, 9000, 20000]
    betas = [0.3, -0.3, 0.0, 0.45, -0.45, 0.2, -0.1, 0.49, -0.49, 0.33]
    out = []
    for nz, v in zip(sizes, betas):
        if interp == w.LAYERS:
            nl = int(rng.integers(1, 12))
            # include narrow layers (down to 2 cells) so a lane sees several boundaries
            widths = rng.integers(2, 60, size=nl - 1) if nl > 1 else np.zeros(0)
            z = rng.uniform(-0.2, 0.5) * nz + np.cumsum(widths) + rng.uniform(0, 1)
            eps = rng.uniform(1.0, 4.0, size=nl)
            mu = rng.uniform(1.0, 1.5, size=nl) if rng.uniform() < 0.5 else np.ones(nl)
        else:
            nk = int(rng.integers(2, 40))
            z = np.sort(rng.uniform(-0.1, 0.9, size=nk)) * nz + np.arange(nk) * 0.7
            eps = rng.uniform(1.0, 4.0, size=nk)
            mu = np.ones(nk)
        srcs = [w.gaussian_source(int(rng.integers(0, nz)), 20.0, 3.0)] if nz > 50 else []
        prbs = [(int(rng.integers(0, nz)), np.linspace(0.1, 0.5, 5))] if nz > 50 else []
        if nz > 50:
            prbs.append((nz - 1, np.linspace(0.2, 0.4, 3)))
        out.append(w.InstanceSpec(nz=nz, beta=v, kind=kind, interp=interp, z=np.asarray(z, float),
                                  eps=eps, mu=mu, sources=srcs, probes=prbs))
    return w.Workload("mixed", 0.5, 0, out)


def storage_round(x, prec):
    """Round on the host to the field storage precision, so both sides start alike."""
    if prec in (gb.F32, gb.F32_KAHAN):
        return x.astype(np.float32).astype(np.float64)
    if prec == gb.F16:
        return x.astype(np.float16).astype(np.float64)
    if prec == gb.BF16:
        import torch
        return torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    return x


def _seed_fields(wl, sim, orcs, seed=11):
    rng = np.random.default_rng(seed)
    for k, I in enumerate(wl.instances):
        B, D = (storage_round(f, sim.prec) for f in w.random_fields(I.nz, rng))
        sim.write_fields(k, gb.FIELD_B, B)
        sim.write_fields(k, gb.FIELD_D, D)
        orcs[k].B[:] = B
        orcs[k].D[:] = D


def _compare(wl, sim, orcs, tol, spectra=True):
    worst = 0.0
    for k, I in enumerate(wl.instances):
        for which, ref in ((gb.FIELD_B, orcs[k].B), (gb.FIELD_D, orcs[k].D)):
            e = rel_l2(sim.read_fields(k, which), ref)
            worst = max(worst, e)
            assert e <= tol, (k, I.nz, I.beta, which, e)
        if spectra:
            for p, (node, om) in enumerate(I.probes):
                e = rel_l2(sim.read_spectrum(k, p, len(om)), orcs[k].spectrum(p))
                worst = max(worst, e)
                assert e <= tol, (k, "probe", p, e)
    return worst


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", [w.PERTURBATION, w.MATTER])
def test_batched_layers_random_fields(shape, kind):
    wl = _mixed_workload(kind=kind)
    sim = make_sim(wl, tuning=shape)
    orcs = make_oracle(wl)
    _seed_fields(wl, sim, orcs)
    n = 3 * shape[1] + 5          # several time blocks and a partial one
    sim.step(n)
    for o in orcs:
        o.run(n)
    assert sim.steps_done() == n
    _compare(wl, sim, orcs, TOL32)


@pytest.mark.parametrize("tuning", [(16, 16), (8, 16), (20, 32), (24, 24)])
@pytest.mark.parametrize("kind", [w.PERTURBATION, w.MATTER])
def test_batched_linear_profiles(kind, tuning):
    wl = _mixed_workload(seed=8, kind=kind, interp=w.LINEAR)
    sim = make_sim(wl, tuning=tuning)
    orcs = make_oracle(wl)
    _seed_fields(wl, sim, orcs)
    sim.step(53)
    for o in orcs:
        o.run(53)
    _compare(wl, sim, orcs, TOL32)


@pytest.mark.parametrize("kind", [w.PERTURBATION, w.MATTER])
def test_plain_kernel_matches_oracle(kind):
    wl = _mixed_workload(seed=9, kind=kind)
    sim = make_sim(wl)
    orcs = make_oracle(wl)
    _seed_fields(wl, sim, orcs)
    sim.step_plain(21)
    for o in orcs:
        o.run(21)
    _compare(wl, sim, orcs, TOL32)


def test_plain_floor_leaves_the_state_alone():
    """gfdtd_plain_floor (the plain path's launches without the arithmetic) leaves
    fields, spectra and the step count as they were, bit for bit."""
    wl = _mixed_workload(seed=12)
    sim = make_sim(wl)
    orcs = make_oracle(wl)
    _seed_fields(wl, sim, orcs)
    sim.step_plain(5)
    before = [(sim.read_fields(k, gb.FIELD_B), sim.read_fields(k, gb.FIELD_D)) for k in range(len(wl.instances))]
    n = sim.steps_done()
    sim.plain_floor(7)
    sim.synchronize()
    assert sim.steps_done() == n
    for k, (B, D) in enumerate(before):
        assert np.array_equal(sim.read_fields(k, gb.FIELD_B), B)
        assert np.array_equal(sim.read_fields(k, gb.FIELD_D), D)


def test_deterministic_and_chunking_independent():
    """The same calls give the same bits; grouping steps into different calls,
    chunks or tile shapes (which moves cells between the fused interior path
    and the edge path) changes results only at the rounding level."""
    wl = _mixed_workload(seed=10)
    res = {}
    for shape, parts in (((16, 16), [1500]), ((16, 16), [1500]), ((16, 16), [700, 3, 797]),
                         ((24, 24), [1500]), ((8, 16), [1024, 476])):
        sim = make_sim(wl, tuning=shape)
        rng = np.random.default_rng(3)
        for k, I in enumerate(wl.instances):
            B, D = (storage_round(f, gb.F32) for f in w.random_fields(I.nz, rng, 1e-3))
            sim.write_fields(k, gb.FIELD_B, B)
            sim.write_fields(k, gb.FIELD_D, D)
        for p in parts:
            sim.step(p)
        res.setdefault((shape, tuple(parts)), []).append(
            [sim.read_fields(k, gb.FIELD_D) for k in range(len(wl.instances))])
    first, again = res[((16, 16), (1500,))]
    for a, b in zip(first, again):
        np.testing.assert_array_equal(a, b)
    for key in (((16, 16), (700, 3, 797)), ((24, 24), (1500,)), ((8, 16), (1024, 476))):
        for a, b in zip(first, res[key][0]):
            assert rel_l2(b, a) <= 1e-5


def test_sources_and_probes_from_rest():
    """Interface workload (Fig. 5 geometry) from zero fields: fields and DFT spectra."""
    wl = w.config1()
    wl.n_steps = 3000
    sim = make_sim(wl)
    orcs = make_oracle(wl)
    sim.step(wl.n_steps)
    orcs[0].run(wl.n_steps)
    _compare(wl, sim, orcs, TOL32)


def test_derived_fields():
    wl = _mixed_workload(seed=12)
    sim = make_sim(wl, tuning=(16, 16))
    orcs = make_oracle(wl)
    _seed_fields(wl, sim, orcs)
    sim.step(40)
    for o in orcs:
        o.run(40)
    for k, I in enumerate(wl.instances):
        n = sim.steps_done()
        eps = orcs[k].material("eps", False, 2 * n + 1)
        mu = orcs[k].material("mu", True, 2 * n)
        E = orcs[k].D / eps
        assert rel_l2(sim.read_fields(k, gb.FIELD_E), E) <= TOL32
        assert rel_l2(sim.read_fields(k, gb.FIELD_H), orcs[k].B / mu) <= TOL32
        Bp = np.concatenate(([0.0, 0.0], orcs[k].B, [0.0]))
        kk = np.arange(I.nz)
        bbar = 0.5 * (Bp[kk + 1] + Bp[kk]) if I.beta >= 0 else 0.5 * (Bp[kk + 2] + Bp[kk + 3])
        assert rel_l2(sim.read_fields(k, gb.FIELD_ESTAR), E - I.beta * bbar) <= TOL32


@pytest.mark.parametrize("kind", [w.PERTURBATION, w.MATTER])
def test_linear_profiles_f64(kind):
    """Piecewise-linear profiles in the FP64 tier, where rounding differences
    between the kernels' per-lane linear pieces and the oracle's per-node
    interpolation would show above the 1e-11 bar if the pieces were wrong."""
    wl = _mixed_workload(seed=8, kind=kind, interp=w.LINEAR)
    sim = make_sim(wl, prec=gb.F64)
    orcs = make_oracle(wl)
    _seed_fields(wl, sim, orcs)
    sim.step(37)
    for o in orcs:
        o.run(37)
    _compare(wl, sim, orcs, 1e-11)


@pytest.mark.parametrize("kind", [w.PERTURBATION, w.MATTER])
def test_f64_four_cell_lanes(kind):
    """The FP64 shape with 4 cells per lane and 8-step time blocks (latency
    shape for small single instances) on ragged layered instances."""
    wl = _mixed_workload(seed=17, kind=kind)
    sim = make_sim(wl, prec=gb.F64, tuning=(4, 8, 4))
    orcs = make_oracle(wl)
    _seed_fields(wl, sim, orcs)
    sim.step(45)
    for o in orcs:
        o.run(45)
    _compare(wl, sim, orcs, 1e-11)


@pytest.mark.parametrize("prec,tol", [(gb.F64, 1e-11), (gb.F32_KAHAN, TOL32), (gb.BF16, 3e-2),
                                      (gb.F16, 5e-3)])
def test_precision_tiers(prec, tol):
    wl = _mixed_workload(seed=13)
    sim = make_sim(wl, prec=prec)
    orcs = make_oracle(wl)
    _seed_fields(wl, sim, orcs)
    sim.step(64)
    for o in orcs:
        o.run(64)
    worst = _compare(wl, sim, orcs, tol, spectra=(prec == gb.F64))
    print("precision tier", prec, "worst relative L2", worst)


@pytest.mark.parametrize("tuning", [None, (20, 24, 7), (24, 24, 6)])
def test_crystal_small_matches_oracle(tuning):
    """Config-3 shape at reduced size (stable velocities), from rest, sources and probes."""
    wl = w.config3(n_inst=48, nz_lo=1 << 10, nz_hi=1 << 13, n_steps=600, stable_only=True)
    sim = make_sim(wl, allow_unstable=False, tuning=tuning)
    orcs = make_oracle(wl)
    sim.step(wl.n_steps)
    import oracle
    oracle.run_many(orcs, wl.n_steps)
    _compare(wl, sim, orcs, TOL32)


@pytest.mark.parametrize("prec,tol", [(gb.F32_KAHAN, TOL32), (gb.F64, 1e-11), (gb.F32, TOL32)])
def test_gradient_ramp_reduced(prec, tol):
    """The moving-gradient shape (linear eps ramp 1 -> 2 over a quarter of the
    grid, v = 0.7c) at 2^12 cells, from rest with its source and probe, long
    enough for the pulse to cross the ramp and reach the probe (8000 smooth
    steps, where FP32 weights that miss a + c = 1 would drift past 1e-4)."""
    wl = w.config4("stable", nz=1 << 12, n_steps=8000)
    sim = make_sim(wl, prec=prec)
    orcs = make_oracle(wl)
    sim.step(wl.n_steps)
    for o in orcs:
        o.run(wl.n_steps)
    _compare(wl, sim, orcs, tol)


def test_gradient_ramp_error_per_tier():
    """The error of every precision tier against the FP64 oracle on the reduced
    moving-gradient run (fields and the probe spectrum, relative L2), printed
    per tier; bounds: FP64 1e-11, Kahan 1e-5, FP32 1e-4, FP16 5e-3, BF16 5e-2
    (measured on GB300: 6e-15, 6.4e-7, 1.8e-6, 1.2e-3, 1.5e-2)."""
    wl = w.config4("stable", nz=1 << 12, n_steps=8000)
    orcs = make_oracle(wl)
    for o in orcs:
        o.run(wl.n_steps)
    bounds = {gb.F64: 1e-11, gb.F32_KAHAN: 1e-5, gb.F32: TOL32, gb.F16: 5e-3, gb.BF16: 5e-2}
    names = {gb.F64: "F64", gb.F32_KAHAN: "F32_KAHAN", gb.F32: "F32", gb.F16: "F16", gb.BF16: "BF16"}
    for prec, bound in bounds.items():
        sim = make_sim(wl, prec=prec)
        sim.step(wl.n_steps)
        eD = rel_l2(sim.read_fields(0, gb.FIELD_D), orcs[0].D)
        eB = rel_l2(sim.read_fields(0, gb.FIELD_B), orcs[0].B)
        eX = rel_l2(sim.read_spectrum(0, 0, len(wl.instances[0].probes[0][1])), orcs[0].spectrum(0))
        print("tier %-9s D %.2e  B %.2e  spectrum %.2e" % (names[prec], eD, eB, eX))
        assert max(eD, eB, eX) <= bound, (names[prec], eD, eB, eX)
        sim.close()


def test_matter_slab_reduced():
    wl = w.config2(velocities=(-0.5, 0.0, 0.5), nz=1 << 13, n_steps=2500)
    sim = make_sim(wl)
    orcs = make_oracle(wl)
    sim.step(wl.n_steps)
    for o in orcs:
        o.run(wl.n_steps)
    _compare(wl, sim, orcs, TOL32)


def test_full_size_crystal_sampled():
    """Config 3 at full size in the benchmark's launch configuration, checked on
    sampled instances that the oracle steps on their own."""
    wl = w.config3(n_steps=64)
    sim = make_sim(wl)
    rng = np.random.default_rng(5)
    sample = sorted(rng.choice(len(wl.instances), size=4, replace=False).tolist())
    start = {}
    for k in sample:
        start[k] = [storage_round(f, gb.F32) for f in w.random_fields(wl.instances[k].nz, rng, 1.0)]
        sim.write_fields(k, gb.FIELD_B, start[k][0])
        sim.write_fields(k, gb.FIELD_D, start[k][1])
    sim.step(wl.n_steps)
    sub = w.Workload("sample", wl.S, wl.n_steps, [wl.instances[k] for k in sample])
    orcs = make_oracle(sub)
    for o, k in zip(orcs, sample):
        o.B[:], o.D[:] = start[k]
    import oracle
    oracle.run_many(orcs, wl.n_steps)
    for o, k in zip(orcs, sample):
        # unstable instances (n|v| > 1) grow, relative error stays relative
        assert rel_l2(sim.read_fields(k, gb.FIELD_D), o.D) <= TOL32
        assert rel_l2(sim.read_fields(k, gb.FIELD_B), o.B) <= TOL32


def test_kahan_reduces_accumulated_rounding():
    """A smooth, finely resolved pulse over many steps: the compensated tier stays
    closer to the FP64 oracle than plain FP32 (the increments per step are small
    next to the fields, where uncompensated FP32 sums lose their low bits)."""
    nz, S, beta, steps = 6000, 0.5, 0.3, 12000
    k = np.arange(nz)
    D0 = np.exp(-((k - 1500) / 300.0) ** 2) * np.cos(2 * np.pi * k / 400.0)
    B0 = D0.copy()
    spec = w.InstanceSpec(nz=nz, beta=beta, z=np.array([4000.0]), eps=np.array([1.0, 2.0]), mu=np.ones(2))
    wl = w.Workload("smooth", S, steps, [spec])
    errs = {}
    for prec in (gb.F32, gb.F32_KAHAN):
        sim = make_sim(wl, prec=prec, tuning=(16, 16))
        Bs, Ds = storage_round(B0, prec), storage_round(D0, prec)
        sim.write_fields(0, gb.FIELD_B, Bs)
        sim.write_fields(0, gb.FIELD_D, Ds)
        o = make_oracle(wl)[0]
        o.B[:], o.D[:] = Bs, Ds
        sim.step(steps)
        o.run(steps)
        errs[prec] = rel_l2(sim.read_fields(0, gb.FIELD_D), o.D)
    print("accumulated rounding: F32 %.3e, F32_KAHAN %.3e" % (errs[gb.F32], errs[gb.F32_KAHAN]))
    assert errs[gb.F32_KAHAN] <= TOL32
    assert errs[gb.F32_KAHAN] < 0.5 * errs[gb.F32]


def _adjoint_workload(n_inst=3, seed=31):
    """Config-5 shape at reduced size: PWL eps over a moving region, transmitted probe."""
    base = w.config5(n_inst=n_inst, nz=1 << 11, n_steps=3400, n_ctrl=48, seed=seed)
    out = []
    for k, I in enumerate(base.instances):
        beta = (0.4, -0.3, 0.25)[k % 3]
        out.append(w.InstanceSpec(nz=I.nz, beta=beta, interp=w.LINEAR, z=I.z - 2046.0 + 600.0,
                                  eps=I.eps, mu=I.mu, sources=[w.gaussian_source(200, 40.0, 3.0)],
                                  probes=[(1300 if beta > 0 else 300, I.probes[0][1])]))
    return w.Workload("adjoint_small", base.S, base.n_steps, out)


def test_adjoint_matches_oracle_adjoint():
    """GPU adjoint (checkpointed, FP32 fields, FP64 gradients) vs the oracle's FP64 adjoint."""
    wl = _adjoint_workload()
    sim = make_sim(wl, allow_unstable=False)
    nv = [len(I.eps) for I in wl.instances]
    loss, grads = sim.adjoint(wl.n_steps, 0, 0, 16, nv)
    assert sim.steps_done() == wl.n_steps
    for k, o in enumerate(make_oracle(wl)):
        L, g = o.adjoint(0, range(16), wl.n_steps)
        assert abs(loss[k] - L) <= 1e-4 * L, (k, loss[k], L)
        assert rel_l2(grads[k], g) <= 1e-3, (k, rel_l2(grads[k], g))
        # the 48 interior controls on their own (the end knots dominate the vector)
        assert rel_l2(grads[k][1:-1], g[1:-1]) <= 1e-3, (k, rel_l2(grads[k][1:-1], g[1:-1]))


def test_adjoint_matches_finite_differences():
    """dL/d(control eps) from the GPU adjoint vs central differences of the FP64
    oracle's loss (h = 1e-4) on a few control points."""
    wl = _adjoint_workload(n_inst=1)
    sim = make_sim(wl, allow_unstable=False)
    loss, grads = sim.adjoint(wl.n_steps, 0, 0, 16, [len(wl.instances[0].eps)])
    I = wl.instances[0]
    import oracle

    def L_of(eps):
        o = oracle.Instance(I.nz, wl.S, I.beta, interp=1, z=I.z, eps=eps, mu=I.mu)
        o.add_source(*I.sources[0])
        o.add_probe(I.probes[0][0], I.probes[0][1])
        o.run(wl.n_steps)
        return float(np.sum(np.abs(o.spectrum(0)) ** 2))

    g = grads[0]
    h = 1e-4
    for j in (3, 17, 30, 44):
        ep, em = I.eps.copy(), I.eps.copy()
        ep[j] += h
        em[j] -= h
        fd = (L_of(ep) - L_of(em)) / (2 * h)
        assert abs(g[j] - fd) <= 1e-3 * np.abs(g).max(), (j, g[j], fd)


def test_adjoint_through_torch_autograd():
    """binding.probe_power as a torch.autograd.Function: the losses equal the
    adjoint's, eps.grad of a weighted sum equals the weighted adjoint
    gradients, and a central difference of the Function's own forward
    (h = 1e-3) matches eps.grad on a control point."""
    torch = pytest.importorskip("torch")
    wl = _adjoint_workload()
    nv = [len(I.eps) for I in wl.instances]

    def make(parts):
        sim = gb.Simulation([I.nz for I in wl.instances], wl.S, gb.F32)
        for k, (I, e) in enumerate(zip(wl.instances, parts)):
            sim.set_medium(k, I.kind, I.beta, I.interp, I.z, e, I.mu, False)
            for s in I.sources:
                sim.add_source(k, *s)
            for p in I.probes:
                sim.add_probe(k, p[0], p[1])
        sim.set_tuning(8, 16, 4)             # the same tiling in every run
        return sim

    eps = torch.tensor(np.concatenate([I.eps for I in wl.instances]), dtype=torch.float64, requires_grad=True)
    loss = gb.probe_power(eps, make, nv, wl.n_steps, 0, 0, 16)
    ref_loss, ref_grads = make([I.eps for I in wl.instances]).adjoint(wl.n_steps, 0, 0, 16, nv)
    assert np.allclose(loss.detach().numpy(), ref_loss, rtol=1e-6, atol=0)
    wts = torch.tensor([1.0, -0.5, 2.0], dtype=torch.float64)
    (loss * wts).sum().backward()
    want = np.concatenate([wk * g for wk, g in zip(wts.numpy(), ref_grads)])
    # (separate runs: FP64 atomics add the gradient in a different order)
    assert rel_l2(eps.grad.numpy(), want) <= 1e-6, rel_l2(eps.grad.numpy(), want)
    j, h = nv[0] + 20, 1e-3                  # a control point of instance 1 (FP32 loss: a wide step)
    with torch.no_grad():
        ep, em = eps.detach().clone(), eps.detach().clone()
        ep[j] += h
        em[j] -= h
        fd = float(((gb.probe_power(ep, make, nv, wl.n_steps, 0, 0, 16)
                     - gb.probe_power(em, make, nv, wl.n_steps, 0, 0, 16)) * wts).sum()) / (2 * h)
    g = eps.grad.numpy()
    assert abs(g[j] - fd) <= 2e-3 * np.abs(g[nv[0]:nv[0] + nv[1]]).max(), (g[j], fd)


def test_profile_kernels_matches_step_and_covers_every_cell():
    """The measurement entry point runs the same launches as step(): identical
    fields and spectra, and its per-kernel cell-updates add up to every cell
    of every instance once per step."""
    wl = w.config3(n_inst=24, nz_lo=1 << 10, nz_hi=1 << 13, n_steps=0, stable_only=True)
    a = make_sim(wl, allow_unstable=False, tuning=(20, 24, 7))
    b = make_sim(wl, allow_unstable=False, tuning=(20, 24, 7))
    n = 1100                       # more than one chunk, ragged last time block
    a.step(n)
    t = b.profile_kernels(n)
    cells = sum(i.nz for i in wl.instances)
    assert sum(v["cell_updates"] for v in t.values()) == cells * n
    assert t["fast"]["launches"] > 0 and t["fast"]["ms"] > 0.0
    for k, inst in enumerate(wl.instances):
        for f in (gb.FIELD_B, gb.FIELD_D):
            assert np.array_equal(a.read_fields(k, f), b.read_fields(k, f))
    assert a.steps_done() == b.steps_done() == n


@pytest.mark.parametrize("tuning", [(24, 24, 6), (20, 16, 7)])
def test_two_boundaries_per_lane_run(tuning):
    """Layers of 14-30 cells under 24-cell lane runs: runs hold two boundaries
    at a time and boundaries pass lane starts in both directions, with sources
    and probes inside the layered region."""
    rng = np.random.default_rng(11)
    out = []
    for v in (0.45, -0.45, 0.2, -0.2, 0.05, -0.33):
        nz = 6000
        widths = rng.integers(14, 31, size=60)
        z = 1500.0 + np.cumsum(widths) + rng.uniform(0, 1)
        eps = np.where(np.arange(len(z) + 1) % 2 == 0, 1.0, rng.uniform(1.5, 3.0))
        out.append(w.InstanceSpec(nz=nz, beta=v, z=z, eps=eps, mu=np.ones(len(eps)),
                                  sources=[w.gaussian_source(1700, 20.0, 3.0)],
                                  probes=[(2000, np.linspace(0.1, 0.5, 5)), (5800, np.linspace(0.2, 0.4, 3))]))
    wl = w.Workload("two_boundaries", 0.5, 700, out)
    sim = make_sim(wl, allow_unstable=False, tuning=tuning)
    st = sim.stats()
    assert (st["cells_per_lane"], st["time_block"]) == tuning[:2]
    orcs = make_oracle(wl)
    sim.step(wl.n_steps)
    for o in orcs:
        o.run(wl.n_steps)
    _compare(wl, sim, orcs, TOL32)
