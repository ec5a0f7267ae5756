"""Batched RAAR (sharp_batch_step): scans of mixed frame size, wrap mode and
frame count stepped together give, scan by scan, the results of stepping
each scan alone with sharp_raar_step (Sec. 2.2 iteration, Eqs. 7-14, with
probe refinement, Eq. 13), on both the recorded-graph and the direct path.

The frame pass of a batch visits the same frames with the same arithmetic;
only the order of the atomic scatter-adds and metric sums differs, so the
two agree to FP32 rounding, not bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu

PROBE_EVERY = 2
RESIDUAL_EVERY = 3
TOL = 2e-5          # relative L2 per step, FP32 rounding of a reordered sum


def _scans():
    out = [synth.scan_batch_member(11, 64, 30), synth.scan_batch_member(12, 128, 12),
           synth.scan_batch_member(13, 64, 17),
           synth.scan_wrapped_raster(seed=14, side=6, m=64, n=128, step=20, photons=1e6),
           synth.scan_batch_member(15, 256, 7), synth.scan_batch_member(16, 256, 4)]
    return out


def _amplitudes(sc):
    rng = np.random.default_rng(sc.seed + 1000)
    inten = O.forward_amplitudes(sc.obj, sc.probe, sc.pos, sc.wrap) ** 2
    return np.sqrt(synth.poisson_intensities(inten, sc.photons, rng)).astype(np.float32)


def _start(S, sc):
    rng = np.random.default_rng(sc.seed + 2000)
    psi0 = synth.random_object(sc.shape, rng, phase_sigma=1.0)
    w0 = synth.perturb_probe(sc.probe, rng, 0.1)
    plan = S.Plan(sc.pos, sc.m, sc.shape, beta=0.75, wrap=sc.wrap, probe_every=PROBE_EVERY,
                  residual_every=RESIDUAL_EVERY)
    plan.raar_init(dev(psi0), dev(w0))
    return plan


def _close(got, ref, floor, it):
    """got matches ref as closely as two runs of the single-scan path match
    each other (the atomics make every run differ at rounding level, and a
    scan with sparse coverage amplifies that over the steps)."""
    err = rel_l2(got, ref)
    return err < max(TOL * it, 16.0 * floor), (err, floor)


def _run(use_graphs, n_steps=8):
    import paper_1602_01448_gb300 as S
    scans = _scans()
    amps = [dev(_amplitudes(sc), torch.float32) for sc in scans]
    alone = [_start(S, sc) for sc in scans]
    again = [_start(S, sc) for sc in scans]     # second single-scan run: the rounding floor
    together = [_start(S, sc) for sc in scans]
    batch = S.Batch(together, amps, use_graphs=use_graphs)
    for it in range(1, n_steps + 1):
        for p, r, a in zip(alone, again, amps):
            p.raar_step(a)
            r.raar_step(a)
        batch.step()
        torch.cuda.synchronize()
        for k, (p, r, q) in enumerate(zip(alone, again, together)):
            for name in ("psi", "c", "probe"):
                ref, got, rep = host(getattr(p, name)), host(getattr(q, name)), host(getattr(r, name))
                ok, info = _close(got, ref, rel_l2(rep, ref), it)
                print(f"step {it} scan {k} {name}: batch {info[0]:.2e} rerun {info[1]:.2e}")
                assert ok, (it, k, name, info)
            mp, mq = host(p.metrics).real, host(q.metrics).real
            np.testing.assert_allclose(mq, mp, rtol=1e-4, atol=1e-7, equal_nan=True, err_msg=f"{it} {k}")
            if it % RESIDUAL_EVERY == 0:
                assert np.all(np.isfinite(mq[:3])), (it, k)
    batch.status()
    for p in together:
        p.status()
    return batch


def test_batch_with_graphs_matches_scans_run_alone():
    batch = _run(True)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for m in (64, 128, 256):
        g = batch.tuned_grid(m)
        assert g > 0 and g % sms == 0, (m, g)
    assert batch.tuned_grid(32) == -1
    batch.close()


def test_batch_direct_path_matches_scans_run_alone():
    _run(False).close()


def test_batch_rebind_drops_recorded_schedules():
    """After new amplitudes are bound the next steps use them (the recorded
    graphs held the old addresses).  A run that kept the old amplitudes ends
    far from the reference (> 10 %); the batch must end within rounding of it
    (the jump in the data makes the rounding differences of the atomics grow
    faster than in the other tests, hence the looser bound)."""
    import paper_1602_01448_gb300 as S
    sc = synth.scan_batch_member(21, 64, 20)
    a1 = dev(_amplitudes(sc), torch.float32)
    a2 = (a1 * 1.5).contiguous()
    p_alone, p_stale, p_batch = _start(S, sc), _start(S, sc), _start(S, sc)
    batch = S.Batch([p_batch], [a1])
    for _ in range(4):
        p_alone.raar_step(a1)
        p_stale.raar_step(a1)
        batch.step()
    batch.amps = [a2]
    S._check(S._C["sharp_batch_bind"](batch.handle, 0, p_batch.c.data_ptr(), p_batch.psi_y.data_ptr(),
                                      p_batch.psi.data_ptr(), p_batch.probe.data_ptr(), a2.data_ptr(),
                                      p_batch.metrics.data_ptr()))
    for _ in range(4):
        p_alone.raar_step(a2)
        p_stale.raar_step(a1)
        batch.step()
    torch.cuda.synchronize()
    ref = host(p_alone.psi)
    assert rel_l2(host(p_stale.psi), ref) > 0.1
    assert rel_l2(host(p_batch.psi), ref) < 1e-2
    batch.close()


def test_batch_rejects_mixed_cadence():
    import paper_1602_01448_gb300 as S
    a = synth.scan_batch_member(31, 64, 9)
    b = synth.scan_batch_member(32, 64, 9)
    pa = _start(S, a)
    pb = S.Plan(b.pos, b.m, b.shape, probe_every=0, residual_every=RESIDUAL_EVERY)
    pb.raar_init(dev(b.psi_init), dev(b.probe_init))
    amps = [dev(_amplitudes(a), torch.float32), dev(_amplitudes(b), torch.float32)]
    with pytest.raises(S.SharpError):
        S.Batch([pa, pb], amps)


def test_every_tuner_candidate_gives_the_same_result():
    """The batch autotuner only changes how frames are scheduled and loaded
    (blocks per SM, rows per round trip of the gathers and the scatter, the
    block-start stagger): every candidate shape steps the scans to the result
    of the default shape within the rounding floor of the atomic sums (two
    runs of the same shape), and the tuner's own choice is one of them."""
    import paper_1602_01448_gb300 as S
    scans = [synth.scan_batch_member(41, 64, 24), synth.scan_batch_member(42, 128, 10),
             synth.scan_batch_member(43, 256, 5)]
    amps = [dev(_amplitudes(sc), torch.float32) for sc in scans]
    plans = [_start(S, sc) for sc in scans]
    batch = S.Batch(plans, amps, use_graphs=False)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n_steps = 2

    def run(shapes):
        for p, sc in zip(plans, scans):
            # restart in the buffers the batch is bound to
            rng = np.random.default_rng(sc.seed + 2000)
            psi0 = dev(synth.random_object(sc.shape, rng, phase_sigma=1.0))
            w0 = dev(synth.perturb_probe(sc.probe, rng, 0.1))
            S.sharp_raar_init(p.handle, psi0, w0, p.c, p.psi_y, p.psi)
            p.probe.copy_(w0)
        for m, shape in shapes.items():
            batch.set_shape(m, *shape)
        batch.iter = 0
        for _ in range(n_steps):
            batch.step()
        batch.status()
        return [host(p.psi) for p in plans]

    default = {64: (sms, 8, 2000), 128: (sms, 8, 2000), 256: (sms, 4, 2000)}
    ref = run(default)
    again = run(default)
    floor = [rel_l2(g, r) for g, r in zip(again, ref)]
    cands = {64: [(k * sms, r, st) for k in (1, 2, 3) for r in (4, 8, 16) for st in (0, 2000)],
             128: [(sms, r, st) for r in (4, 8, 16) for st in (0, 2000)],
             256: [(sms, r, st) for r in (2, 4) for st in (0, 2000)]}
    for m, shapes in cands.items():
        for shape in shapes:
            got = run({**default, m: shape})
            k = [sc.m for sc in scans].index(m)
            err = rel_l2(got[k], ref[k])
            assert err < max(TOL * n_steps, 16.0 * floor[k]), (m, shape, err, floor[k])
    with pytest.raises(S.SharpError):
        batch.set_shape(256, sms, 8, 0)           # 8 rows: not a 256^2 candidate
    with pytest.raises(S.SharpError):
        batch.set_shape(32, sms, 8, 0)            # no scan of that size
    batch.close()

    # a fresh batch picks one of the candidates (tuned now, or earlier in the
    # process for its frame size and size class)
    plans2 = [_start(S, sc) for sc in scans]
    b2 = S.Batch(plans2, amps, use_graphs=True)
    for _ in range(8):
        b2.step()
    b2.status()
    for m, shapes in cands.items():
        shape = b2.tuned_shape(m)
        assert shape in shapes, (m, shape)
    b2.close()
