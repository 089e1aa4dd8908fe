"""The autotuner on the GPU: a real search over (skin, lanes per atom) on a
small Lennard-Jones batch, the cache hit on the second call, and that the
tuned settings give the same forces as the defaults (the tunables change the
schedule, not the result)."""
import numpy as np
import pytest

from _helpers import lj_cell
from paper_1902_09171_gb300 import autotune, rcell

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


def test_tune_searches_caches_and_keeps_results(torch, tmp_path):
    cells = [lj_cell(6, seed=k) for k in range(4)]
    st = torch.cuda.Stream()
    path = str(tmp_path / "cache.json")
    make = lambda skin: rcell.params_lj_cu(skin=skin)
    best, hit = autotune.tune(make, cells, st, skins=(0.5, 1.0), tpas=(1, 2), n_steps=20, path=path)
    assert not hit
    assert best["skin"] in (0.5, 1.0) and best["tpa"] in (1, 2) and best["ms_per_step"] > 0
    assert len(best["table"]) >= 2
    assert min(r["ms_per_step"] for r in best["table"]) == best["ms_per_step"]
    again, hit2 = autotune.tune(make, cells, st, skins=(0.5, 1.0), tpas=(1, 2), n_steps=20, path=path)
    assert hit2 and again["skin"] == best["skin"] and again["tpa"] == best["tpa"]

    # the tuned schedule gives the forces of the default one (summation order aside)
    forces = []
    for skin, tpa in ((1.0, 1), (best["skin"], best["tpa"])):
        ctx = rcell.rcell_create(make(skin), cells)
        try:
            rcell.rcell_set_tuning(ctx, tpa, 1)
            rcell.rcell_eval(ctx)
            assert rcell.rcell_sync(ctx) == 0
            forces.append(np.concatenate([rcell.rcell_get_atoms(ctx, k, len(c["x0"]))[2] for k, c in enumerate(cells)]))
        finally:
            rcell.rcell_destroy(ctx)
    f0, f1 = forces
    scale = np.sqrt((f0[:, :3] ** 2).sum(1).mean())
    assert np.abs(f0[:, :3] - f1[:, :3]).max() <= 1e-5 * scale
