"""The training driver: JSON-lines metrics (loss terms, throughput, test error
against the exact Poisson solution) and checkpoint / resume continuing the
same step numbering and optimiser state."""
import numpy as np
import pytest

from paper_2409_14248_gb300 import build, capi, inputs, trainer

pytestmark = pytest.mark.gpu

pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    capi.load_library()


def test_trainer_logs_json_lines(tmp_path):
    log = str(tmp_path / "run.jsonl")
    with trainer.Trainer("poisson_2_5_1") as tr:
        recs = tr.run(300, log_path=log, log_every=100)
    back = trainer.read_log(log)
    assert back == recs
    assert [r["step"] for r in back] == [100, 200, 300]
    for r in back:
        assert set(r) == {"step", "loss", "loss_pde", "loss_bnd", "ms_per_step", "points_per_s", "test_rel_l2"}
        assert np.isfinite(r["loss"]) and r["points_per_s"] > 0 and r["ms_per_step"] > 0
        assert r["loss"] == pytest.approx(inputs.WORKLOADS["poisson_2_5_1"].alpha * r["loss_pde"] + r["loss_bnd"])
    assert back[-1]["loss"] < back[0]["loss"]
    assert back[-1]["test_rel_l2"] < back[0]["test_rel_l2"]


def test_trainer_resume_continues_the_run(tmp_path):
    ck = str(tmp_path / "run.ck")
    with trainer.Trainer("poisson_2_5_1", flags=capi.HRKAN_FLAG_LAYERWISE) as a:
        a.run(200, log_every=100, checkpoint_path=ck, checkpoint_every=100)
    with trainer.Trainer("poisson_2_5_1", flags=capi.HRKAN_FLAG_LAYERWISE) as b:
        b.resume(ck)
        assert b.t == 200
        rb = b.run(100, log_every=100)
        Wb = b.W.cpu().numpy()
    with trainer.Trainer("poisson_2_5_1", flags=capi.HRKAN_FLAG_LAYERWISE) as c:
        rc = c.run(300, log_every=100)
        Wc = c.W.cpu().numpy()
    assert rb[-1]["step"] == rc[-1]["step"] == 300
    # the layer-wise path reduces in a fixed order: the resumed run is the same run
    assert Wb.tobytes() == Wc.tobytes()
    assert rb[-1]["loss"] == rc[-1]["loss"]
