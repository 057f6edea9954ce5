"""Serving (continuous batching) and the plain FP32 comparator, on the GPU,
through the C ABI.  Each request's result must equal its result alone
(bitwise), whatever it was batched with."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_13925_gb300 import channels as C

from gpu_util import rel_fro, run, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_13925_gb300 import build
    build.build()
    return torch


def _pool(torch, insts, T=6, tol=0.0):
    from paper_2305_13925_gb300 import binding
    Hd = [to_dev(i.H, torch) for i in insts]
    Wd = [to_dev(np.zeros(i.H.shape), torch) for i in insts]
    descs = [binding.instance(Hd[k], Wd[k], insts[k].xi, T, tol) for k in range(len(insts))]
    return Hd, Wd, descs


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
def test_server_results_equal_alone(torch_gpu, precision):
    torch = torch_gpu
    from paper_2305_13925_gb300 import binding
    insts = C.generate_ragged(24, 51, k_set=(8, 32, 64, 128), m_set=(256, 512, 1024))
    alone = [run([i.H], [i.xi], T=6, precision=precision)["W"][0] for i in insts]
    Hd, Wd, descs = _pool(torch, insts)
    prec = binding.Precoder(max_instances=64, max_M=1024, max_K=128, precision=precision)
    srv = binding.jacpcg_server_create(prec.ctx, max_batch=8, max_inflight=3)
    try:
        tickets = [binding.jacpcg_submit(srv, d) for d in descs]
        res = [binding.jacpcg_poll(srv, t) for t in tickets]
        assert all(r[0] == 0 for r in res) and all(r[1] > 0 for r in res)
        n_done, n_batches, mean_b = binding.jacpcg_server_stats(srv)
        assert n_done == len(insts) and n_batches >= 3
    finally:
        binding.jacpcg_server_destroy(srv)
        prec.close()
    torch.cuda.synchronize()
    for k, i in enumerate(insts):
        W = Wd[k].T.cpu().numpy().astype(np.complex128)
        assert np.array_equal(W, alone[k]), k


@pytest.mark.parametrize("policy", ["cost_class", "fifo"])
def test_server_cost_classes(torch_gpu, policy):
    """Requests of the 64 class, of the 256 class with M >= 4 K and of the
    near-square 256 class: under the cost-class policy no batch mixes
    classes (so at least three batches run); under FIFO any mix may share a
    batch.  Either way each result equals the request's result alone."""
    torch = torch_gpu
    from paper_2305_13925_gb300 import binding
    insts = (C.generate_ragged(4, 81, k_set=(64,), m_set=(256,))
             + C.generate_ragged(2, 82, k_set=(256,), m_set=(1024,))
             + C.generate_ragged(2, 83, k_set=(256,), m_set=(512,)))
    order = [0, 4, 6, 1, 5, 2, 7, 3]                       # classes interleaved in arrival order
    insts = [insts[k] for k in order]
    runs = [run([i.H], [i.xi], T=12, tol=1e-5, precision="tf32x3") for i in insts]
    alone = [r["W"][0] for r in runs]
    alone_status = [int(r["status"][0]) for r in runs]   # near-square channels may stop unconverged
    Hd, Wd, descs = _pool(torch, insts, T=12, tol=1e-5)
    prec = binding.Precoder(max_instances=16, max_M=1024, max_K=256, precision="tf32x3")
    pol = binding.JACPCG_BATCH_COST_CLASS if policy == "cost_class" else binding.JACPCG_BATCH_FIFO
    srv = binding.jacpcg_server_create(prec.ctx, max_batch=16, max_inflight=2, batch_policy=pol)
    try:
        tickets = [binding.jacpcg_submit(srv, d) for d in descs]
        res = [binding.jacpcg_poll(srv, t) for t in tickets]
        n_done, n_batches, _ = binding.jacpcg_server_stats(srv)
    finally:
        binding.jacpcg_server_destroy(srv)
        prec.close()
    assert [r[0] for r in res] == alone_status and n_done == len(insts)
    if policy == "cost_class":
        assert n_batches >= 3
    torch.cuda.synchronize()
    for k in range(len(insts)):
        assert np.array_equal(Wd[k].T.cpu().numpy().astype(np.complex128), alone[k]), k


def test_server_replay_poisson_trace(torch_gpu):
    torch = torch_gpu
    from paper_2305_13925_gb300 import binding
    insts = C.generate_ragged(32, 61, k_set=(16, 64), m_set=(256, 1024))
    Hd, Wd, descs = _pool(torch, insts)
    rng = np.random.default_rng(4)
    n_req = 400
    arrivals = np.cumsum(rng.exponential(1e6 / 20000.0, n_req))      # 20k requests/s
    which = np.arange(n_req) % len(insts)
    prec = binding.Precoder(max_instances=256, max_M=1024, max_K=64, precision="tf32x3")
    srv = binding.jacpcg_server_create(prec.ctx, max_batch=128, max_inflight=4)
    try:
        lat, st = binding.jacpcg_server_replay(srv, descs, which, arrivals)
    finally:
        binding.jacpcg_server_destroy(srv)
        prec.close()
    assert (st == 0).all()
    assert (lat > 0).all() and np.median(lat) < 1e5
    torch.cuda.synchronize()
    for k in (0, 5, 17):
        ref = O.precode(C.round_complex64(insts[k].H), insts[k].xi, "standard", max_iter=6)["W"]
        assert rel_fro(Wd[k].T.cpu().numpy().astype(np.complex128), ref) <= 1e-5


def test_server_admission_with_small_arena(torch_gpu):
    """An arena that holds only a few instances: the server launches smaller
    batches and waits for memory, results stay exact; a request larger than
    the whole arena is refused with ENOMEM."""
    torch = torch_gpu
    from paper_2305_13925_gb300 import binding
    insts = C.generate_ragged(10, 71, k_set=(64,), m_set=(512,))
    Hd, Wd, descs = _pool(torch, insts)
    alone = [run([i.H], [i.xi], T=6)["W"][0] for i in insts]
    big = C.generate_ragged(1, 72, k_set=(256,), m_set=(512,))[0]
    Hb, Wb, db = _pool(torch, [big])
    prec = binding.Precoder(max_instances=16, max_M=512, max_K=256, arena_bytes=3 * 70 * 1024)
    srv = binding.jacpcg_server_create(prec.ctx, max_batch=16, max_inflight=2)
    try:
        tickets = [binding.jacpcg_submit(srv, d) for d in descs]
        tb = binding.jacpcg_submit(srv, db[0])
        res = [binding.jacpcg_poll(srv, t) for t in tickets]
        rb = binding.jacpcg_poll(srv, tb)
        n_done, n_batches, mean_b = binding.jacpcg_server_stats(srv)
    finally:
        binding.jacpcg_server_destroy(srv)
        prec.close()
    assert all(r[0] == 0 for r in res)
    assert rb[0] == binding.JACPCG_ENOMEM
    assert n_batches >= 4                           # at most 3 instances fit at once
    torch.cuda.synchronize()
    for k in range(len(insts)):
        assert np.array_equal(Wd[k].T.cpu().numpy().astype(np.complex128), alone[k])


@pytest.mark.parametrize("variant", ["standard", "cg"])
def test_plain_comparator_parity(torch_gpu, variant):
    torch = torch_gpu
    from paper_2305_13925_gb300 import binding
    H, xi = C.generate_batch("batched_1024x64", 6, 1)
    insts = [C.Instance(C.round_complex64(h), x, 0.0, None) for h, x in zip(H, xi)]
    insts += C.generate_ragged(3, 81, k_set=(17, 100), m_set=(256,))
    Hd, Wd, descs = _pool(torch, insts)
    ws = torch.empty(binding.plain_workspace_bytes(128), dtype=torch.uint8, device="cuda")
    status = torch.full((len(insts),), -1, dtype=torch.int32, device="cuda")
    beta = torch.zeros(len(insts), dtype=torch.float32, device="cuda")
    binding.jacpcg_precode_plain(descs, ws, variant, status, None, None, beta,
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    for k, i in enumerate(insts):
        ref = O.precode(C.round_complex64(i.H), i.xi, variant, max_iter=6)
        W = Wd[k].T.cpu().numpy().astype(np.complex128)
        bar = 1e-5 if variant == "standard" else 1e-3
        assert rel_fro(W, ref["W"]) <= bar, (k, rel_fro(W, ref["W"]))
        assert abs(beta[k].item() - ref["beta"]) <= 1e-4 * ref["beta"]
