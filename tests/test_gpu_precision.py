"""Precision sweep over a velocity ensemble: snapshot storage FP32 / BF16 /
FP16 (per-snapshot max-abs scaling) x imaging interval 1 / 4 / 8, FP32 wave
stepping, Kahan FP32 stacking, FP64 ensemble statistics.  Images and
standard-deviation maps from the GPU (rtm_migrate_ensemble +
rtm_ensemble_stats) against the FP64 oracle with the same quantisation
replayed, and against exact snapshots.

Sizes are scaled down from the 1701 x 351 x 5000 ensemble so that the
oracle finishes in seconds: 16 samples of a layered model (201 x 101 cells at
10 m, 4 % Gaussian-random-field perturbation, water fixed) x 2 shots x 800
steps.
"""
import numpy as np
import pytest

import oracle
from conftest import rel_l2
from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NS, NX, NZ, NT = 16, 201, 101, 800
IMG_TOL = {rtm.SNAP_F32: 1e-3, rtm.SNAP_BF16: 1e-2, rtm.SNAP_F16: 1e-2}
STD_TOL = 2e-2


@pytest.fixture(scope="module")
def problem():
    base = inputs.layered_faulted(NZ, NX, 10.0, 10.0, seed=404, water_depth=100.0)
    ens = inputs.ensemble(base, 10.0, 10.0, NS, water_depth=100.0).astype(np.float32)
    s = inputs.Survey(NX, NZ, 20, 10.0, 10.0, 1e-3, NT, base, np.array([50, 150], np.int32),
                      np.array([1, 1], np.int32), np.arange(NX, dtype=np.int32),
                      np.full(NX, 1, np.int32), inputs.ricker(15.0, 1e-3, NT))
    g = oracle.grid(*s.grid_tuple())
    w = s.wavelet.astype(np.float32).astype(np.float64)
    data = np.stack([oracle.model(g, base.astype(np.float32).astype(np.float64), s.src_ix[k],
                                  s.src_iz[k], s.rec_ix, s.rec_iz, w) for k in range(2)])
    return s, ens, data.astype(np.float32), g, w


def _oracle_images(s, ens, data, g, w, isnap, mode):
    return np.stack([oracle.migrate(g, ens[i].astype(np.float64), s.src_ix, s.src_iz, s.rec_ix,
                                    s.rec_iz, w, data.astype(np.float64), isnap=isnap,
                                    snap_mode=mode) for i in range(NS)])


@pytest.fixture(scope="module")
def ctx():
    c = rtm.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("isnap", [1, 4, 8])
def test_precision_sweep(ctx, problem, isnap):
    s, ens, data, g, w = problem
    exact = _oracle_images(s, ens, data, g, w, isnap, 0)
    _, exact_std, _, _ = oracle.ensemble_stats(exact.reshape(NS, -1))
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    report = {}
    for mode in (rtm.SNAP_F32, rtm.SNAP_BF16, rtm.SNAP_F16):
        imgs = torch.zeros((NS, NZ, NX), dtype=torch.float32, device="cuda")
        ctx.migrate_ensemble(rtm.make_grid(*s.grid_tuple()), torch.from_numpy(ens).cuda(), acq,
                             torch.from_numpy(data).cuda(), rtm.Opts(isnap, mode, 1e-6, 1), imgs)
        outs = [torch.zeros(NZ * NX, dtype=t, device="cuda")
                for t in (torch.float64, torch.float64, torch.float32, torch.float32)]
        ctx.ensemble_stats(imgs, *outs)
        torch.cuda.synchronize()
        got = imgs.cpu().numpy()
        got_std = outs[1].cpu().numpy()
        want = exact if mode == rtm.SNAP_F32 else _oracle_images(s, ens, data, g, w, isnap, mode)
        _, want_std, _, _ = oracle.ensemble_stats(want.reshape(NS, -1))
        e_img = max(rel_l2(got[i], want[i]) for i in range(NS))
        e_std = rel_l2(got_std, want_std)
        x_img = max(rel_l2(got[i], exact[i]) for i in range(NS))
        x_std = rel_l2(got_std, exact_std)
        report[mode] = (e_img, e_std, x_img, x_std)
        # against the oracle with the same snapshot format
        assert e_img <= IMG_TOL[mode], (mode, isnap, e_img)
        assert e_std <= STD_TOL, (mode, isnap, e_std)
    # against exact snapshots: FP16 within the half-precision bounds at every
    # interval; BF16 only at isnap 1 (its 8-bit significand exceeds 1e-2 at
    # isnap >= 4 once the Laplacian filter amplifies the quantisation noise)
    assert report[rtm.SNAP_F16][2] <= 1e-2 and report[rtm.SNAP_F16][3] <= 2e-2, report
    if isnap == 1:
        assert report[rtm.SNAP_BF16][2] <= 1e-2 and report[rtm.SNAP_BF16][3] <= 2e-2, report
    print(f"isnap {isnap}: " + ", ".join(
        f"{['f32', 'bf16', 'f16'][m]} img {r[0]:.2e}/{r[2]:.2e} std {r[1]:.2e}/{r[3]:.2e}"
        for m, r in report.items()))


def test_full_size_half_precision_parity(ctx):
    """Half-precision snapshots at the full 1701 x 351, 5000-step size
    (isnap 4), where per-snapshot max scaling meets the 10 Hz fields' full
    dynamic range.  One shot migrated with FP16 and with BF16 snapshots
    against the oracle replaying the same quantisation (1e-2), its error
    against exact snapshots reported; then the std map of 4 velocity samples
    x that shot in each format against the oracle's std map (2e-2)."""
    s = inputs.full_size(nshot=96)
    shot = 47
    one = inputs.Survey(s.nx, s.nz, s.nb, s.dx, s.dz, s.dt, s.nt, s.vel, s.src_ix[shot:shot + 1],
                        s.src_iz[shot:shot + 1], s.rec_ix, s.rec_iz, s.wavelet)
    g = oracle.grid(*one.grid_tuple())
    w = one.wavelet.astype(np.float32).astype(np.float64)
    data = oracle.model(g, s.vel.astype(np.float32).astype(np.float64), one.src_ix[0],
                        one.src_iz[0], one.rec_ix, one.rec_iz, w).astype(np.float32)[None]
    vm = inputs.smooth(s.vel, s.dx, s.dz, 60.0).astype(np.float32)
    ens = inputs.ensemble(vm, s.dx, s.dz, 4).astype(np.float32)
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, one.src_ix, one.src_iz, one.rec_ix, one.rec_iz,
                       one.wavelet.astype(np.float32))
    grid = rtm.make_grid(*one.grid_tuple())

    def ora(vel, mode):
        return oracle.migrate(g, vel.astype(np.float64), one.src_ix, one.src_iz, one.rec_ix,
                              one.rec_iz, w, data.astype(np.float64), isnap=4, snap_mode=mode)

    exact = ora(vm, 0)
    report = {}
    for mode in (rtm.SNAP_F16, rtm.SNAP_BF16):
        img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
        ctx.migrate(grid, torch.from_numpy(vm).cuda(), acq, torch.from_numpy(data).cuda(),
                    rtm.Opts(4, mode, 1e-6, 1), img)
        imgs = torch.zeros((4, s.nz, s.nx), dtype=torch.float32, device="cuda")
        ctx.migrate_ensemble(grid, torch.from_numpy(ens).cuda(), acq,
                             torch.from_numpy(data).cuda(), rtm.Opts(4, mode, 1e-6, 1), imgs)
        outs = [torch.zeros(s.nz * s.nx, dtype=t, device="cuda")
                for t in (torch.float64, torch.float64, torch.float32, torch.float32)]
        ctx.ensemble_stats(imgs, *outs)
        torch.cuda.synchronize()
        got = img.cpu().numpy()
        want = ora(vm, mode)
        _, want_std, _, _ = oracle.ensemble_stats(
            np.stack([ora(ens[i], mode) for i in range(4)]).reshape(4, -1))
        e_img = rel_l2(got, want)
        e_std = rel_l2(outs[1].cpu().numpy(), want_std)
        report[mode] = (e_img, rel_l2(got, exact), e_std, rel_l2(want, exact))
        assert e_img <= IMG_TOL[mode], (mode, e_img)
        assert e_std <= STD_TOL, (mode, e_std)
    print("full size, isnap 4: " + ", ".join(
        f"{['f32', 'bf16', 'f16'][m]} img {r[0]:.2e} vs replay / {r[1]:.2e} vs exact "
        f"(oracle replay vs exact {r[3]:.2e}), std {r[2]:.2e}" for m, r in report.items()))
