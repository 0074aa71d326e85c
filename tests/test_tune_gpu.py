"""Autotuner (alp_tune through the C-ABI): exhaustive sweep, database, cache,
timing proxy, prediction, and what the learned cost model gains over tuning
without it."""
import json
import os

import numpy as np
import pytest

from paper_1706_10086_gb300 import inputs, tuning

pytestmark = pytest.mark.gpu


def test_exhaustive_sweep_db_and_lookup(alp, tmp_path):
    db = str(tmp_path / "db.jsonl")
    os.environ["ALP_TUNE_DB"] = db
    os.environ["ALP_TUNE_RUNS"] = "2"
    try:
        alp.alp_tune_clear_cache()
        st, cfg, tf = alp.alp_tune(300, 200, 100, alp.ALP_PATH_NATIVE, alp.ALP_TUNE_EXHAUSTIVE)
        assert alp.alp_config_valid(cfg) and tf > 0
        recs = tuning.load_db(db)
        assert len(recs) == 1 and recs[0]["M"] == 300 and recs[0]["path"] == "native"
        rows = recs[0]["configs"]
        assert len(rows) == alp.alp_config_count(alp.ALP_PATH_NATIVE)
        est = [r[6] for r in rows]
        assert tuple(rows[recs[0]["winner"]][:6]) == cfg.astuple()
        assert min(est) == est[recs[0]["winner"]]
        st, cfg2, _ = alp.alp_tune(300, 200, 100, alp.ALP_PATH_NATIVE, alp.ALP_TUNE_LOOKUP)
        assert cfg2.astuple() == cfg.astuple()
        st, _, _ = alp.alp_tune(301, 200, 100, alp.ALP_PATH_NATIVE, alp.ALP_TUNE_LOOKUP,
                                raise_on_error=False)
        assert st == alp.ALP_ERR_NOT_TUNED
        st, ecfg, _ = alp.alp_tune(256, 512, 300, alp.ALP_PATH_EMUL, alp.ALP_TUNE_EXHAUSTIVE)
        assert alp.alp_config_valid(ecfg, alp.ALP_PATH_EMUL)
        assert tuning.load_db(db)[-1]["path"] == "emul"
        # resume: collect skips what is present
        assert tuning.collect([(300, 200, 100)], ["native"], db) == 0
    finally:
        os.environ.pop("ALP_TUNE_DB", None)
        alp.alp_tune_clear_cache()


def test_timing_proxy_tracks_full_runs(alp):
    """The one-wave, K <= 256 proxy against whole-problem timings."""
    for (M, N, K) in [(2048, 2048, 1024), (4096, 1024, 2048), (1000, 3000, 700)]:
        for cfg in [(128, 128, 16, 8, 8, 0), (64, 64, 16, 4, 4, 0)]:
            est = alp.alp_tune_time_config(M, N, K, alp.ALP_PATH_NATIVE, cfg, True, 3)
            full = alp.alp_tune_time_config(M, N, K, alp.ALP_PATH_NATIVE, cfg, False, 2)
            assert abs(est / full - 1) < 0.15, (M, N, K, cfg, est, full)


def test_emulated_proxy_ranks_like_full_runs(alp):
    """The emulated timing proxy (K capped at 2048) against whole-problem
    timings: within 20 %, and it ranks the CTA-pair config above the
    one-block config as the full runs do."""
    E = alp.ALP_PATH_EMUL
    single, pair = (128, 256, 64, 1, 0, 8), (256, 256, 64, 2, 0, 16)
    for (M, N, K) in [(4096, 4096, 4096), (2048, 8192, 4096)]:
        est = {c: alp.alp_tune_time_config(M, N, K, E, c, True, 3) for c in (single, pair)}
        full = {c: alp.alp_tune_time_config(M, N, K, E, c, False, 2) for c in (single, pair)}
        for c in (single, pair):
            assert abs(est[c] / full[c] - 1) < 0.2, (M, N, K, c, est[c], full[c])
        assert (est[pair] < est[single]) == (full[pair] < full[single]), (est, full)


def test_predict_needs_model(alp):
    alp.alp_tune_unload_model()
    st, _, _ = alp.alp_tune(512, 512, 512, alp.ALP_PATH_NATIVE, alp.ALP_TUNE_PREDICT,
                            raise_on_error=False)
    assert st == alp.ALP_ERR_NOT_TUNED


def test_learned_model_beats_tuning_without_it(alp, tmp_path):
    """Reduced version of the predictor workload (shapes log-uniform in
    [64, 16384], both paths): sweep 400 training and 100 held-out shapes, train
    the MLP on the GPU, and compare the regret of its choices on the held-out
    (shape, path) cases with the two ways of choosing without it: one config
    per path tuned once at N = 10240 (the paper's protocol, Sect. 3 and
    Table 4) and the winner of the nearest training shape.  The network must
    have a lower mean and a lower 90th-percentile regret than both."""
    db = str(tmp_path / "db.jsonl")
    seed = inputs.workload_seed("mlp_predictor")
    train_sh = inputs.shapes(seed + 200, 400, 64, 16384)
    test_sh = inputs.shapes(seed + 300, 100, 64, 16384)
    tuning_shape = (10240, 10240, 10240)
    paths = ["native", "emul"]
    tuning.collect(train_sh, paths, db, runs=2)
    tuning.collect(test_sh, paths, db, runs=2)
    tuning.collect([tuning_shape], paths, db, runs=2)
    recs = tuning.load_db(db)
    key = lambda r: (r["M"], r["N"], r["K"])
    train_keys = {tuple(int(v) for v in s) for s in train_sh}
    test_keys = {tuple(int(v) for v in s) for s in test_sh} - train_keys
    train_ds = tuning.dataset([r for r in recs if key(r) in train_keys])
    test_ds = tuning.dataset([r for r in recs if key(r) in test_keys])
    tuning_ds = tuning.dataset([r for r in recs if key(r) == tuning_shape])
    model, hist = tuning.train(train_ds, epochs=3000, lr=3e-3)
    assert hist[-1] < hist[0]
    res = tuning.evaluate(model, train_ds, test_ds, tuning_ds=tuning_ds)
    print(json.dumps(res))
    mlp = res["mlp"]
    for other in ("fixed_tuned_once", "nearest_shape"):
        assert mlp["mean"] < res[other]["mean"], (other, res)
        assert mlp["p90"] < res[other]["p90"], (other, res)
    # the model drives PREDICT and cfg == NULL calls
    params, mean, std = model
    alp.alp_tune_load_model(params, train_ds["C"], mean, std)
    try:
        st, cfg, _ = alp.alp_tune(700, 300, 900, alp.ALP_PATH_NATIVE, alp.ALP_TUNE_PREDICT)
        assert alp.alp_config_valid(cfg)
        st, cfg, _ = alp.alp_tune(700, 300, 900, alp.ALP_PATH_EMUL, alp.ALP_TUNE_PREDICT)
        assert alp.alp_config_valid(cfg, alp.ALP_PATH_EMUL)
    finally:
        alp.alp_tune_unload_model()
