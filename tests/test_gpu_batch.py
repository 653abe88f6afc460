"""GPU parity of the batch of realisations (pm_batch_*): every realisation of a batched,
graph-replayed run matches the same run done alone, and the FP64 oracle."""
import numpy as np
import pytest

from oracle import cic, ic, pm as opm, stats
from oracle.cosmology import Cosmology
from tests.gpu_util import lib, min_image, positions_box_units, rel_l2, ticks_to_host, to_host, torch

pytestmark = pytest.mark.gpu

BOXES = [1000.0, 2000.0, 4000.0]
SEEDS = [11, 12, 13]
NP, NMESH, A_I, A_F, STEPS = 32, 64, 0.1, 1.0, 6


def _cfg(pm, box=1000.0):
    return pm.make_config(NP, NMESH, box, A_I, A_F, STEPS)


def _single(pm, box, seed, steps):
    run = pm.PMRun(_cfg(pm, box))
    run.ic(seed=seed)
    run.step(steps)
    x, p = run.particles()
    torch.cuda.synchronize()
    return ticks_to_host(x).copy(), to_host(p).astype(np.float64).copy()


def _batch_particles(b, r):
    x, p = b.particles(r)
    torch.cuda.synchronize()
    return ticks_to_host(x).copy(), to_host(p).astype(np.float64).copy()


def _disp(x, x0):
    return min_image(positions_box_units(x) - positions_box_units(x0))


@pytest.mark.parametrize("graph", [True, False])
def test_batched_runs_match_single_runs(graph):
    pm = lib()
    b = pm.PMBatch(_cfg(pm), boxes=BOXES)
    b.ic(SEEDS)
    x0 = [_batch_particles(b, r)[0] for r in range(3)]
    b.step(2, graph=graph)      # first segment (includes the initial deposit)
    b.step(STEPS - 2, graph=graph)
    assert b.state() == (STEPS, pytest.approx(A_F, abs=1e-15), True)
    for r, (box, seed) in enumerate(zip(BOXES, SEEDS)):
        xs, ps = _single(pm, box, seed, STEPS)
        xb, pb = _batch_particles(b, r)
        # same kernels and parameters; only the order of FP32 atomic additions differs
        assert rel_l2(_disp(xb, x0[r]), _disp(xs, x0[r])) < 1e-5
        assert rel_l2(pb, ps) < 1e-5


def test_graph_replay_is_reused_and_matches_direct_launches():
    pm = lib()
    out = []
    for graph in (True, False):
        b = pm.PMBatch(_cfg(pm), boxes=BOXES)
        for rep in range(2):  # the second run from step 0 replays the cached graph
            b.ic(SEEDS)
            b.step(STEPS, graph=graph)
        out.append([_batch_particles(b, r) for r in range(3)])
    for r in range(3):
        assert rel_l2(out[0][r][1], out[1][r][1]) < 1e-5


def test_batched_power_matches_oracle_and_single_runs():
    pm = lib()
    b = pm.PMBatch(_cfg(pm), boxes=BOXES)
    b.ic(SEEDS)
    b.step(STEPS)
    edges = stats.log_edges(8, 1.0, NMESH / 2.0)
    k, p, nm = b.power(edges)
    c = Cosmology()
    for r in (0, 2):
        x0, p0 = ic.zeldovich(c, NP, BOXES[r], A_I, seed=SEEDS[r], fixed=True)
        ref = opm.PMRun(c, NMESH, BOXES[r], A_I, A_F, STEPS, x0, p0)
        ref.step(STEPS)
        ko, po, no = stats.power_spectrum(cic.density_contrast(ref.x, NMESH), BOXES[r], edges)
        np.testing.assert_array_equal(nm[r], no)
        ok = no > 0
        assert np.max(np.abs(p[r][ok] / po[ok] - 1)) < 1e-3
        np.testing.assert_allclose(k[r][ok], ko[ok], rtol=1e-12)


def test_growth_matched_stepping_in_a_batch_matches_single_runs():
    pm = lib()
    cfg = pm.make_config(NP, NMESH, BOXES[0], A_I, A_F, STEPS, stepping=pm.PM_STEP_GROWTH)
    b = pm.PMBatch(cfg, boxes=BOXES)
    b.ic(SEEDS)
    b.step(STEPS, graph=True)
    for r, (box, seed) in enumerate(zip(BOXES, SEEDS)):
        run = pm.PMRun(pm.make_config(NP, NMESH, box, A_I, A_F, STEPS, stepping=pm.PM_STEP_GROWTH))
        run.ic(seed=seed)
        x0 = ticks_to_host(run.particles()[0]).copy()
        run.step(STEPS)
        xs, ps = ticks_to_host(run.particles()[0]).copy(), to_host(run.particles()[1]).astype(np.float64)
        xb, pb = _batch_particles(b, r)
        assert rel_l2(_disp(xb, x0), _disp(xs, x0)) < 1e-5
        assert rel_l2(pb, ps) < 1e-5


def test_batched_bias_matches_single_pipeline():
    pm = lib()
    b = pm.PMBatch(_cfg(pm), boxes=BOXES)
    b.ic(SEEDS)
    b.step(STEPS)
    edges = stats.log_edges(10, 1.0, NMESH / 2.0)
    coef = b.bias(edges, k_max=0.05, terms=2)
    for r in range(3):
        run = pm.PMRun(_cfg(pm, BOXES[r]))
        run.ic(seed=SEEDS[r])
        run.step(STEPS)
        dm = run.density()
        dh = torch.empty_like(dm)
        pm.pm_halo_proxy(run.ctx, dh, field=dm)
        want, _, _, _ = pm.pm_linear_bias(run.ctx, dh, dm, edges, 0.05, terms=2)
        np.testing.assert_allclose(coef[r], want, rtol=1e-3)
        assert coef[r][0] > 1.0  # the densest cells are a positively biased tracer


def test_batched_paired_fixed_ics_match_the_oracle():
    # the IC flags reach every realisation: paired-and-fixed phases of each seed, each box
    pm = lib()
    b = pm.PMBatch(_cfg(pm), boxes=BOXES)
    b.ic(SEEDS, paired=True, fixed=True)
    c = Cosmology()
    for r, (box, seed) in enumerate(zip(BOXES, SEEDS)):
        xb, pb = _batch_particles(b, r)
        xo, po = ic.zeldovich(c, NP, box, A_I, seed=seed, paired=True, fixed_amplitude=True)
        q = ic.lattice_ticks(NP)
        assert rel_l2(_disp(xb, q), _disp(xo, q)) < 2e-6
        assert rel_l2(pb, po) < 2e-6


def test_batched_2lpt_ics_match_the_oracle():
    pm = lib()
    b = pm.PMBatch(_cfg(pm), boxes=BOXES)
    b.ic(SEEDS, lpt_order=2)
    c = Cosmology()
    for r, (box, seed) in enumerate(zip(BOXES, SEEDS)):
        xb, pb = _batch_particles(b, r)
        xo, po = ic.zeldovich(c, NP, box, A_I, seed=seed, lpt_order=2)
        q = ic.lattice_ticks(NP)
        assert rel_l2(_disp(xb, q), _disp(xo, q)) < 2e-6
        assert rel_l2(pb, po) < 2e-6


@pytest.mark.parametrize("chunk", [1, 2])
@pytest.mark.parametrize("graph", [True, False])
def test_chunked_batch_matches_whole_batch(chunk, graph):
    # realisations per launch change only the launch shape (chunk 2 of 3 leaves a partial chunk)
    pm = lib()
    out = []
    for c in (0, chunk):
        b = pm.PMBatch(_cfg(pm), boxes=BOXES)
        b.set_chunk(c)
        b.ic(SEEDS)
        b.step(STEPS, graph=graph)
        out.append([_batch_particles(b, r) for r in range(3)])
    for r in range(3):
        q = ic.lattice_ticks(NP)
        assert rel_l2(_disp(out[1][r][0], q), _disp(out[0][r][0], q)) < 1e-6
        assert rel_l2(out[1][r][1], out[0][r][1]) < 1e-6


def test_autotuned_batch_matches_single_runs():
    pm = lib()
    b = pm.PMBatch(_cfg(pm), boxes=BOXES)
    chunk, ms = b.autotune()
    assert chunk in (3, 2, 1) and ms > 0
    b.ic(SEEDS)
    b.step(STEPS)
    for r, (box, seed) in enumerate(zip(BOXES, SEEDS)):
        xs, ps = _single(pm, box, seed, STEPS)
        xb, pb = _batch_particles(b, r)
        q = ic.lattice_ticks(NP)
        assert rel_l2(_disp(xb, q), _disp(xs, q)) < 1e-5
        assert rel_l2(pb, ps) < 1e-5
    with pytest.raises(pm.PMError) as e:
        b.autotune()  # the run has started
    assert e.value.status == 7
    b2 = pm.PMBatch(_cfg(pm), boxes=BOXES)
    b2.ic(SEEDS)
    with pytest.raises(pm.PMError) as e:
        b2.autotune()  # would overwrite the ICs
    assert e.value.status == 7
    with pytest.raises(pm.PMError):
        b.set_chunk(4)


def test_whole_plane_form_of_the_batch_matches_the_separate_passes():
    # 64 x 128^3 is the batched workload's mesh; here three realisations on 128^3 meshes with the
    # middle FFT passes on whole kz planes in shared memory (form 1) and as separate launches
    pm = lib()
    cfg = pm.make_config(32, 128, 1000.0, A_I, A_F, STEPS)
    out = []
    for form in (0, 1):
        b = pm.PMBatch(cfg, boxes=BOXES)
        b.set_fft(form)
        assert b.tuning() == (3, form)
        b.ic(SEEDS)
        b.step(STEPS, graph=True)
        out.append([_batch_particles(b, r) for r in range(3)])
        del b
    for (xs, ps), (xp, pp) in zip(*out):
        assert rel_l2(pp, ps) < 1e-5
        assert np.max(np.abs(_disp(xp, xs))) < 1e-5


def test_batch_autotuner_picks_a_form_and_chunk():
    pm = lib()
    b = pm.PMBatch(pm.make_config(32, 128, 1000.0, A_I, A_F, STEPS), boxes=BOXES * 2)
    chunk, ms = b.autotune()
    c2, form = b.tuning()
    assert c2 == chunk and chunk in (6, 3, 2, 1) and form in (0, 1) and ms > 0
    b.ic(SEEDS * 2)
    b.step(STEPS, graph=True)
    assert b.state()[0] == STEPS


def test_batched_bispectrum_ratio_matches_single_pipeline():
    # Sec. 5.3 on the batched ensemble: per realisation (its context view) the density, the halo
    # proxy and B_hhh / B_mmm on the equilateral and squeezed (k3 = 4 k_f) slices, against the same
    # pipeline on the realisation run alone (which test_gpu_bias.py checks against the oracle)
    pm = lib()
    b = pm.PMBatch(_cfg(pm), boxes=BOXES)
    b.ic(SEEDS)
    b.step(STEPS)
    edges = np.arange(0.5, 16.0, 1.0)
    nb = len(edges) - 1
    eq, sq = pm.bispectrum_configurations(nb, 3)
    for r in range(3):
        dm = b.density(r)
        dh = torch.empty_like(dm)
        pm.pm_halo_proxy(b.context(r), dh, field=dm)
        bh, ntri = b.bispectrum(r, edges, 64, field=dh)
        bm, _ = b.bispectrum(r, edges, 64, field=dm)
        run = pm.PMRun(_cfg(pm, BOXES[r]))
        run.ic(seed=SEEDS[r])
        run.step(STEPS)
        dm1 = run.density()
        dh1 = torch.empty_like(dm1)
        pm.pm_halo_proxy(run.ctx, dh1, field=dm1)
        bh1, ntri1 = run.bispectrum(edges, 64, field=dh1)
        bm1, _ = run.bispectrum(edges, 64, field=dm1)
        np.testing.assert_array_equal(ntri, ntri1)
        for sl in (eq, sq):
            idx = np.asarray(sl)
            ok = ntri[idx] > 0
            assert np.count_nonzero(ok) > 3
            np.testing.assert_allclose(bm[idx][ok], bm1[idx][ok], rtol=1e-4, atol=1e-6 * np.max(np.abs(bm1[idx])))
            np.testing.assert_allclose((bh / bm)[idx][ok], (bh1 / bm1)[idx][ok], rtol=1e-3)


@pytest.mark.parametrize("n_lo,graph", [(0, True), (4, True), (4, False)])
def test_poisson_gauge_batch_matches_single_runs(n_lo, graph):
    # the Poisson gauge in a batch (per-realisation Phi history and FP64 island, boxes of 2, 8
    # and 20 Gpc/h where the lag matters): every realisation equals the run done alone, and the
    # batch's realisation on the largest box equals the oracle's Poisson-gauge run
    pm = lib()
    boxes, seeds, steps = [2000.0, 8000.0, 20000.0], [21, 22, 23], 8
    cfg = pm.make_config(NP, NMESH, boxes[0], 0.02, 1.0, steps, mode=1, n_lo=n_lo)
    b = pm.PMBatch(cfg, boxes=boxes)
    b.ic(seeds)
    b.step(steps, graph=graph)
    assert b.state()[0] == steps and b.state()[2]
    for r in range(3):
        run = pm.PMRun(pm.make_config(NP, NMESH, boxes[r], 0.02, 1.0, steps, mode=1, n_lo=n_lo))
        run.ic(seed=seeds[r])
        x0 = ticks_to_host(run.particles()[0]).copy()
        run.step(steps)
        xs, ps = ticks_to_host(run.particles()[0]).copy(), to_host(run.particles()[1]).astype(np.float64)
        xb, pb = _batch_particles(b, r)
        assert rel_l2(_disp(xb, x0), _disp(xs, x0)) < 1e-5
        assert rel_l2(pb, ps) < 1e-5
    c = Cosmology()
    x0, p0 = ic.zeldovich(c, NP, boxes[2], 0.02, seed=seeds[2], fixed=True)
    ref = opm.PMRun(c, NMESH, boxes[2], 0.02, 1.0, steps, x0, p0, mode=opm.GR_POISSON)
    ref.step(steps)
    xb, pb = _batch_particles(b, 2)
    assert rel_l2(_disp(xb, x0), _disp(ref.x, x0)) < 2e-3
