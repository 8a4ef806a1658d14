"""The serving form: continuous batching with admission by device memory.

Frames submitted from several client threads while batches are on the GPU
are encoded in shared batches; each result must equal the frame encoded
alone (fv_encode_batch_bf16 on that frame only) within 1e-5 and the FP64
oracle on the same bf16 input within 2e-3. Admission refuses frames once the
HBM budget or the slots are used up and admits them again after results are
polled; unknown tickets and non-blocking polls report their statuses."""
import threading

import numpy as np
import pytest

from gpu_util import TOL, case, max_err, oracle_fv, torch_cuda
from paper_1604_03498_gb300 import fv, synth

pytestmark = pytest.mark.gpu
P = fv.FV_PREC_BF16


def _alone(g, X):
    torch = torch_cuda()
    Xd = torch.from_numpy(X).cuda()
    out = torch.zeros(1, 2 * g.K * g.D, device="cuda")
    fv.fv_encode_batch(g, Xd, [0, X.shape[0]], out)
    torch.cuda.synchronize()
    return out.cpu().numpy()[0]


def test_server_results_equal_alone_and_in_the_mix():
    torch_cuda()
    K, D = 128, 64
    _, w, mu, var = case(K, D, 10, 60)
    g = fv.fv_gmm_load(w, mu, var, P)
    # a 50 ms batching window makes frames submitted close together share batches
    srv = fv.fv_server_create(g, max_slots=256, hbm_budget_bytes=1 << 30, max_batch_descriptors=200000,
                              max_batch_frames=64, max_frame_descriptors=40000, batch_window_ns=50_000_000)
    rng = np.random.default_rng(3)
    sizes = [[int(rng.integers(1, 9000)) if j % 4 else int(rng.integers(20000, 40000)) for j in range(12)]
             for _ in range(4)]
    data = [[synth.sample_descriptors(w, mu, var, n, seed=1000 * c + j, gmm_frac=0.8) for j, n in enumerate(sz)]
            for c, sz in enumerate(sizes)]
    frames = {}
    lock = threading.Lock()

    def client(cid):
        for X in data[cid]:
            st, t = fv.fv_server_submit(srv, cid, X)
            with lock:
                frames[t] = (cid, X)

    threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    batch_sizes = []
    for i, (t, (cid, X)) in enumerate(sorted(frames.items())):
        out = np.zeros(2 * K * D, np.float32)
        st, info = fv.fv_server_poll(srv, t, out, timeout_ns=10_000_000_000)
        assert st == fv.FV_OK and info["stream_id"] == cid and info["n"] == X.shape[0]
        assert info["latency_ns"] > 0 and info["queue_ns"] >= 0
        batch_sizes.append(info["batch_frames"])
        assert max_err(out, _alone(g, X)) <= 1e-5
        if i % 8 == 0:
            assert max_err(out, oracle_fv(synth.to_bf16_grid(X), w, mu, var)) <= TOL[P]
    stats = fv.fv_server_stats(srv)
    assert stats["completed"] == len(frames) == 48
    assert max(batch_sizes) > 1          # frames did share batches
    srv.close()
    g.close()


def test_server_admission_by_memory_and_statuses():
    torch_cuda()
    K, D = 64, 32
    _, w, mu, var = case(K, D, 10, 61)
    g = fv.fv_gmm_load(w, mu, var, P)
    n = 10000
    frame_bytes = n * D * 4
    srv = fv.fv_server_create(g, max_slots=8, hbm_budget_bytes=2 * frame_bytes, max_batch_descriptors=50000,
                              max_batch_frames=8, max_frame_descriptors=40000)
    X = synth.sample_descriptors(w, mu, var, n, seed=7, gmm_frac=0.8)
    _, t1 = fv.fv_server_submit(srv, 0, X)
    _, t2 = fv.fv_server_submit(srv, 0, X)
    refused = 0
    # a third frame fits only once earlier frames have finished
    st, t3 = fv.fv_server_submit(srv, 0, X, allow=(fv.FV_OK, fv.FV_ERR_BUSY))
    refused += st == fv.FV_ERR_BUSY
    out = np.zeros(2 * K * D, np.float32)
    for t in (t1, t2):
        st, info = fv.fv_server_poll(srv, t, out, timeout_ns=10_000_000_000)
        assert st == fv.FV_OK
    if refused:
        st, t3 = fv.fv_server_submit(srv, 0, X)
    st, info = fv.fv_server_poll(srv, t3, out, timeout_ns=10_000_000_000)
    assert st == fv.FV_OK
    assert max_err(out, _alone(g, X)) <= 1e-5
    stats = fv.fv_server_stats(srv)
    assert stats["refused"] == refused and stats["completed"] == 3
    with pytest.raises(fv.FVError) as e:
        fv.fv_server_poll(srv, 123456, out, timeout_ns=0)
    assert e.value.status == fv.FV_ERR_NOTFOUND
    with pytest.raises(fv.FVError) as e:
        fv.fv_server_poll(srv, t3, out, timeout_ns=0)   # already released
    assert e.value.status == fv.FV_ERR_NOTFOUND
    with pytest.raises(fv.FVError) as e:
        fv.fv_server_submit(srv, 0, np.zeros((50000, D), np.float32))
    assert e.value.status == fv.FV_ERR_INVALID
    _, t4 = fv.fv_server_submit(srv, 1, X)
    st, _ = fv.fv_server_poll(srv, t4, out, timeout_ns=0)
    assert st in (fv.FV_PENDING, fv.FV_OK)
    if st == fv.FV_PENDING:
        st, _ = fv.fv_server_poll(srv, t4, out, timeout_ns=10_000_000_000)
        assert st == fv.FV_OK
    srv.close()
    g.close()
