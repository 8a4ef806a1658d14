"""The batched form: a plan with one captured CUDA graph per batch.

Checks that a graph launch over a ragged batch (an empty frame, a 1-row
frame, frames ending inside 128-row tiles and 64-row stages) gives the same
vectors as the direct BF16 path and stays within 2e-3 of the FP64 oracle on
the same bf16 input; that a second batch with other sizes and fewer frames
replays the same graph correctly (no stale state); and that the autotune
writes its choice to the cache and a later plan reads it back."""
import os

import numpy as np
import pytest

from gpu_util import TOL, case, max_err, oracle_fv, torch_cuda
from paper_1604_03498_gb300 import fv, synth

pytestmark = pytest.mark.gpu
P = fv.FV_PREC_BF16


def _batch(w, mu, var, sizes, seed):
    frames = [synth.sample_descriptors(w, mu, var, n, seed=seed + i, gmm_frac=0.8) for i, n in enumerate(sizes)]
    offs = np.zeros(len(sizes) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    return frames, offs


def test_plan_graph_matches_direct_path_and_oracle(tmp_path):
    torch = torch_cuda()
    K, D = 256, 64
    _, w, mu, var = case(K, D, 10, 50)
    g = fv.fv_gmm_load(w, mu, var, P)
    cache = str(tmp_path / "tune.txt")
    plan = fv.fv_batch_plan_create(g, max_frames=8, max_rows=60000, autotune=True, tune_cache=cache)
    info = fv.fv_batch_plan_get_info(plan)
    assert info["tuned"] == 1 and info["stat_ctas"] >= 1
    assert info["rows_per_tile"] == 128 and info["y_stages"] in (1, 2) and info["candidates"] >= 4
    for sizes, seed in (([5000, 0, 12000, 1, 20001, 129], 600), ([777, 30000], 700)):
        frames, offs = _batch(w, mu, var, sizes, seed)
        X = torch.from_numpy(np.concatenate([f for f in frames if len(f)], 0)).cuda()
        out = torch.full((len(sizes), 2 * K * D), float("nan"), device="cuda")
        assert fv.fv_batch_plan_run_f32(plan, X, offs, out) == fv.FV_OK
        ref = torch.full((len(sizes), 2 * K * D), float("nan"), device="cuda")
        fv.fv_encode_batch(g, X, offs, ref)
        torch.cuda.synchronize()
        o, r = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert max_err(o, r) <= 1e-5
        for f, row in zip(frames, o):
            if len(f) == 0:
                assert np.all(row == 0)
            elif len(f) in (1, 129, 777):
                assert max_err(row, oracle_fv(synth.to_bf16_grid(f), w, mu, var)) <= TOL[P]
    plan.close()
    # a second plan with the same key reads the tuned grid back
    plan2 = fv.fv_batch_plan_create(g, max_frames=8, max_rows=60000, autotune=True, tune_cache=cache)
    info2 = fv.fv_batch_plan_get_info(plan2)
    assert info2["tuned"] == 2 and info2["stat_ctas"] == info["stat_ctas"] and info2["y_stages"] == info["y_stages"]
    assert os.path.exists(cache)
    plan2.close()
    g.close()


def test_plan_bf16_input_and_host_output():
    torch = torch_cuda()
    K, D = 64, 32
    _, w, mu, var = case(K, D, 10, 51)
    g = fv.fv_gmm_load(w, mu, var, P)
    plan = fv.fv_batch_plan_create(g, max_frames=4, max_rows=10000)
    frames, offs = _batch(w, mu, var, [300, 4000, 2], 800)
    Xf = np.concatenate(frames, 0)
    Xb = torch.from_numpy(Xf).cuda().to(torch.bfloat16)
    fv.fv_batch_plan_load_bf16(plan, Xb, D, int(offs[-1]))
    out = np.full((3, 2 * K * D), np.nan, np.float32)
    assert fv.fv_batch_plan_run(plan, offs, out) == fv.FV_OK
    for f, row in zip(frames, out):
        assert max_err(row, oracle_fv(synth.to_bf16_grid(f), w, mu, var)) <= TOL[P]
    with pytest.raises(fv.FVError) as e:
        fv.fv_batch_plan_run(plan, np.array([0, 20000], np.int64))
    assert e.value.status == fv.FV_ERR_INVALID
    plan.close()
    g.close()


def test_plan_full_size_batch_of_256_frames_matches_oracle(tmp_path):
    """The batched workload at full size: 256 frames, N ~ Uniform{5000..40000}
    (5.84 M rows), one graph launch; six sampled frames (the smallest, the
    largest and four seeded others) against the oracle on their bf16 rows.
    Frame contents are rows gathered from a 16-frame pool (as in the bench)."""
    torch = torch_cuda()
    K, D, B = 256, 64, 256
    _, w, mu, var = case(K, D, 10, 52)
    pool = np.concatenate([synth.sample_descriptors(w, mu, var, 40000, seed=900 + i, gmm_frac=0.8)
                           for i in range(16)])
    sizes = synth.frame_sizes(B, 5000, 40000, seed=4)
    offs = np.zeros(B + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    rows = int(offs[-1])
    src = (np.arange(rows, dtype=np.int64) * 7919) % pool.shape[0]
    g = fv.fv_gmm_load(w, mu, var, P)
    plan = fv.fv_batch_plan_create(g, max_frames=B, max_rows=rows, autotune=True,
                                   tune_cache=str(tmp_path / "tune.txt"))
    poolb = torch.from_numpy(pool).cuda().to(torch.bfloat16)
    fv.fv_batch_plan_load_bf16(plan, poolb[torch.from_numpy(src).cuda()], D, rows)
    out = torch.full((B, 2 * K * D), float("nan"), device="cuda")
    assert fv.fv_batch_plan_run(plan, offs, out) == fv.FV_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes))} |
                  {int(i) for i in np.random.default_rng(52).choice(B, 4, replace=False)})
    poolr = synth.to_bf16_grid(pool)
    for b in pick:
        Xf = poolr[src[offs[b]:offs[b + 1]]]
        assert max_err(got[b], oracle_fv(Xf, w, mu, var)) <= TOL[P], b
    plan.close()
    g.close()
