"""The surrogate's MD fallback on the GPU (fe_step_surrogate) against the
oracle's reading of it (oracle/fallback.py).

Floating point decides the integer flags here, so the decision is compared on
the GPU's own FP32 spread: the oracle decides on the spread the GPU reported
and the flags must agree bit for bit.  The spread itself is compared with the
oracle's ensemble statistics of its own FP64 member predictions (exact for
members whose output is their bias, BF16 tolerance for general members), and
the stress handed to the FE update with the oracle's merge.

A point that comes back to MD after frozen increments replays the increments
it missed, one by one, from its frozen r-cell state; its stress is compared with
an all-MD run of the same cells along the same deformation path.
"""
import numpy as np
import pytest

import oracle
from _helpers import lj_cell
from oracle import fallback as fb
from oracle import mlp
from paper_1902_09171_gb300 import inputs, pipeline, rcell
from paper_1902_09171_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    t.cuda.set_device(0)
    from paper_1902_09171_gb300 import build
    build.build()
    rcell.load()
    return t


def bf16(a):
    x = np.asarray(a, dtype=np.float32).copy()
    u = x.view(np.uint32)
    u += ((u >> 16) & 1) + np.uint32(0x7FFF)
    u &= np.uint32(0xFFFF0000)
    return x.astype(np.float64)


def bf16_weights(theta):
    p = mlp.unpack(theta)
    for k in ("W1", "W2", "W3", "W4"):
        p[k] = bf16(p[k])
    return mlp.pack(p)


class Bar:
    """A 4-element bar of 256-atom LJ r-cells with a K-member surrogate, all on one stream."""

    def __init__(self, torch, K, ne=4, seed=10):
        self.t = torch
        self.st = torch.cuda.Stream()
        torch.cuda.set_stream(self.st)
        prm = rcell.params_lj_cu()
        cells = [lj_cell(4, seed=seed + k) for k in range(ne)]
        L = cells[0]["H0"][0, 0]
        X, conn = inputs.hex_mesh(ne, 1, 1, ne * L, L, L)
        mask, val = inputs.uniaxial_bc(X, ne * L)
        self.ne, self.K = ne, K
        self.ctx = rcell.rcell_create(prm, cells, stream=self.st)
        self.fe = rcell.fe_create(X, conn, mask, val, 0.3, 0.05, 20.0, 0.0, stream=self.st)
        self.sur = S.sur_create(K, ne, 1, 3, stream=self.st)
        dev = torch.device("cuda")
        self.h = torch.zeros((K, ne, 128), dtype=torch.float32, device=dev)
        self.Fp = torch.eye(3, dtype=torch.float64, device=dev).repeat(ne, 1, 1).contiguous()
        self.flag = torch.zeros(ne, dtype=torch.int32, device=dev)
        self.spread = torch.zeros(ne, dtype=torch.float32, device=dev)
        self.P = torch.zeros((ne, 3, 3), dtype=torch.float64, device=dev)

    def step(self, lam, on, off, s_floor, force):
        prev = self.flag.cpu().numpy().copy()
        n = rcell.fe_step_surrogate(self.fe, self.ctx, self.sur, lam, 20, 10, on, off, s_floor, int(force), self.h,
                                    self.Fp, self.flag, self.spread)
        rcell.fe_get_P(self.fe, self.P)
        self.t.cuda.synchronize()
        return (n, prev, self.flag.cpu().numpy().copy(), self.spread.cpu().numpy().astype(np.float64),
                self.Fp.cpu().numpy().copy(), self.P.cpu().numpy().copy())

    def close(self):
        rcell.fe_destroy(self.fe)
        rcell.rcell_destroy(self.ctx)
        S.sur_destroy(self.sur)
        self.t.cuda.set_stream(self.t.cuda.default_stream())


def bias_only(member_out):
    """Parameters of a member whose every output is its head bias: all weights and the
    hidden biases zero, b4[0:6] = member_out."""
    p = mlp.unpack(np.zeros(mlp.N_PARAMS))
    p["b4"][:6] = member_out
    return mlp.pack(p).astype(np.float32)


def test_scripted_spreads_trip_hold_and_release_like_the_oracle(torch):
    # four members at m + d (+1, +1, -1, -1) on sigma_xx: the spread is 2 d / sqrt(3) / |m|,
    # scripted increment by increment across the trip and release thresholds
    K, on, off, s_floor = 4, 0.02, 0.01, 1e-3
    m = np.array([1.5, 0.25, 0.25, 0.0, 0.0, 0.0])
    script = [0.005, 0.03, 0.004, 0.03, 0.015, 0.012, 0.009, 0.015, 0.025, 0.0]
    bar = Bar(torch, K)
    try:
        for k, target in enumerate(script):
            d = target * np.linalg.norm(m) * np.sqrt(3.0) / 2.0
            outs = [m + d * np.array([s, 0, 0, 0, 0, 0]) for s in (1, 1, -1, -1)]
            for j in range(K):
                S.sur_set_params(bar.sur, j, bias_only(outs[j]))
            force = k < 2
            n, prev, flag, spread, F, P = bar.step(0.001 * (k + 1), on, off, s_floor, force)
            # the oracle's member predictions (FP64 forward of the same parameters)
            pred = np.array([mlp.forward(bias_only(o).astype(np.float64), np.zeros((bar.ne, 1, 15)))[0][:, 0]
                             for o in outs])
            mean, sp = fb.ensemble_stats(pred, s_floor)
            assert np.abs(spread - sp).max() <= 1e-4 * sp.max() + 1e-7, (k, spread, sp)
            want = fb.decide(spread, prev, on, off, force)
            assert np.array_equal(flag, want), (k, flag, want, spread)
            assert n == int((want != 0).sum())
            # the stress of the FE update: the surrogate's P = J sigma F^-T where not on MD
            for e in range(bar.ne):
                if flag[e] == 0:
                    ref = fb.cauchy_to_pk1(F[e], mean[e])
                    assert np.abs(P[e] - ref).max() <= 1e-6 * np.abs(ref).max()
        assert rcell.rcell_sync(bar.ctx) == 0
    finally:
        bar.close()


def test_ensemble_of_trained_shape_members_decides_like_the_oracle(torch):
    # general members (seeded weights): per-point spreads differ; the thresholds follow
    # the previous increment's spreads (on at their median, off at half of it) on
    # increments 2, 3, 5, 6 so that points trip and hold, and are lifted out of
    # reach on increments 4 and 7 so that every point is released
    K, s_floor = 4, 0.05
    thetas = [mlp.init_params(60 + k).astype(np.float32) for k in range(K)]
    bar = Bar(torch, K, ne=6, seed=30)
    try:
        for j in range(K):
            S.sur_set_params(bar.sur, j, thetas[j])
        Fs, spreads, flags, prevs, ons, offs, forces, Ps = [], [], [], [], [], [], [], []
        on, off = 1e9, 1e9
        for k in range(8):
            force = k < 2
            n, prev, flag, spread, F, P = bar.step(0.002 * (k + 1), on, off, s_floor, force)
            Fs.append(F)
            spreads.append(spread)
            flags.append(flag)
            prevs.append(prev)
            ons.append(on)
            offs.append(off)
            forces.append(force)
            Ps.append(P)
            assert n == int((flag != 0).sum())
            if k in (3, 6):
                on = off = 1e9
            else:
                on = float(np.quantile(spread, 0.5))
                off = 0.5 * on
        assert rcell.rcell_sync(bar.ctx) == 0
    finally:
        bar.close()
    # the oracle: features of the F history, each member's recurrence, ensemble stats
    F_hist = np.stack(Fs, axis=1)  # (ne, T, 3, 3)
    ne, T = F_hist.shape[:2]
    U = np.zeros((ne, T, 15))
    Fprev = np.tile(np.eye(3), (ne, 1, 1))
    for t in range(T):
        U[:, t] = mlp.features(Fprev, F_hist[:, t])
        Fprev = F_hist[:, t]
    pred = np.array([mlp.forward(bf16_weights(th.astype(np.float64)), bf16(U))[0] for th in thetas])  # K, ne, T, 6
    n_trip = 0
    for t in range(T):
        mean, sp = fb.ensemble_stats(pred[:, :, t], s_floor)
        assert np.abs(spreads[t] - sp).max() <= 5e-2 * max(sp.max(), 1e-3) + 2e-3, (t, spreads[t], sp)
        want = fb.decide(spreads[t], prevs[t], ons[t], offs[t], forces[t])
        assert np.array_equal(flags[t], want), (t, flags[t], want)
        n_trip += int((want == 1).sum())
        for e in range(ne):
            if want[e] == 0:
                ref = fb.cauchy_to_pk1(Fs[t][e], mean[e])
                assert np.abs(Ps[t][e] - ref).max() <= 5e-2 * max(np.abs(ref).max(), 1e-3)
    assert n_trip > 0 and sum(int((f == 0).sum()) for f in flags[2:]) > 0


def test_point_returning_to_md_replays_its_missed_increments(torch):
    # Kremer-Grest glass r-cells (Sec. 3.2's material) behind a bar whose every node is
    # prescribed, so that F follows the load alone: bar A runs the surrogate with
    # scripted spreads (MD forced for 2 increments, surrogate for 3, then a trip back
    # to MD), bar B runs all-MD (fe_step) on the same cells with the same seeds.  On
    # its return every point of A replays the three missed increments from its frozen
    # state, so its r-cells follow B's deformation path step by step, with B's Philox
    # counters: the stress that A hands to the FE equals B's to rounding.
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    ne, K, n_steps, n_avg = 4, 4, 200, 100
    try:
        ctx0, cells = pipeline.prepare_kg_batch(ne, n_chains=40, chain_len=50, seed=71, stream=st,
                                                soft_steps=1500, eq_steps=1000)
        rcell.rcell_destroy(ctx0)
        L = cells[0]["H0"][0, 0]
        X, conn = inputs.hex_mesh(ne, 1, 1, ne * L, L, L)
        mask, val = inputs.uniaxial_bc(X, ne * L, all_nodes=True)
        prm = rcell.params_kg(seed=5)
        ca, cb = rcell.rcell_create(prm, cells, stream=st), rcell.rcell_create(prm, cells, stream=st)
        fa = rcell.fe_create(X, conn, mask, val, 0.85, 0.05, 1.0, 0.0, stream=st)
        fb_ = rcell.fe_create(X, conn, mask, val, 0.85, 0.05, 1.0, 0.0, stream=st)
        sur = S.sur_create(K, ne, 1, 3, stream=st)
        dev = torch.device("cuda")
        h = torch.zeros((K, ne, 128), dtype=torch.float32, device=dev)
        Fp = torch.eye(3, dtype=torch.float64, device=dev).repeat(ne, 1, 1).contiguous()
        flag = torch.zeros(ne, dtype=torch.int32, device=dev)
        Pa = torch.zeros((ne, 3, 3), dtype=torch.float64, device=dev)
        Pb = torch.zeros((ne, 3, 3), dtype=torch.float64, device=dev)
        m = np.array([1.0, 0.5, 0.5, 0.0, 0.0, 0.0])
        try:
            script = [0.001, 0.001, 0.001, 0.001, 0.001, 0.05]  # spreads; 0, 1 forced
            for k, target in enumerate(script):
                d = target * np.linalg.norm(m) * np.sqrt(3.0) / 2.0
                for j, sgn in enumerate((1, 1, -1, -1)):
                    S.sur_set_params(sur, j, bias_only(m + d * np.array([sgn, 0, 0, 0, 0, 0])))
                lam = 0.01 * (k + 1)
                n, rep = rcell.fe_step_surrogate(fa, ca, sur, lam, n_steps, n_avg, 0.02, 0.01, 1e-3, k < 2, h, Fp,
                                                 flag, with_replays=True)
                rcell.fe_step(fb_, cb, lam, n_steps, n_avg, None)
                rcell.fe_get_P(fa, Pa)
                rcell.fe_get_P(fb_, Pb)
                torch.cuda.synchronize()
                want_n, want_rep = {0: (ne, 0), 1: (ne, 0), 5: (ne, 3 * ne)}.get(k, (0, 0))
                assert (n, rep) == (want_n, want_rep), (k, n, rep)
                if n == ne:
                    a, b = Pa.cpu().numpy(), Pb.cpu().numpy()
                    assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max(), (k, np.abs(a - b).max())
            assert rcell.rcell_sync(ca) == 0 and rcell.rcell_sync(cb) == 0
        finally:
            for fe in (fa, fb_):
                rcell.fe_destroy(fe)
            for c in (ca, cb):
                rcell.rcell_destroy(c)
            S.sur_destroy(sur)
    finally:
        torch.cuda.set_stream(torch.cuda.default_stream())
