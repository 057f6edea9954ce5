"""jacpcg_precode_noalloc, the entry point for callers that cannot allocate
(real-time slot loops that forbid allocator latency, integrations whose
memory was fixed at start-up).  It must give the same precoders as
jacpcg_precode within the W tolerance, call after call, while using only its
static device scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2305_13925_gb300 import channels as C

pytestmark = pytest.mark.gpu

TOL_W = 1e-5


@pytest.fixture(scope="module")
def torch_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_13925_gb300 import build
    build.build()
    return torch


def _batch(torch):
    from paper_2305_13925_gb300 import binding
    H, xi = C.generate_batch("batched_1024x64", 12, 41)
    Hs = list(H) + [i.H for i in C.generate_ragged(3, 42, k_set=(8, 100, 256), m_set=(256, 1024))]
    xis = list(xi) + [i.xi for i in C.generate_ragged(3, 42, k_set=(8, 100, 256), m_set=(256, 1024))]
    Hd, Wd = [], []
    for h in Hs:
        M, K = h.shape
        ld = M + (M & 1)
        t = torch.zeros((K, ld), dtype=torch.complex64)
        t[:, :M] = torch.from_numpy(np.ascontiguousarray(h.T).astype(np.complex64))
        Hd.append(t.cuda()[:, :M])
        Wd.append(torch.zeros((K, ld), dtype=torch.complex64, device="cuda")[:, :M])
    insts = [binding.instance(Hd[i], Wd[i], xis[i], 6) for i in range(len(Hs))]
    return Hd, Wd, insts


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_precode_on_two_calls(torch_gpu):
    torch = torch_gpu
    from paper_2305_13925_gb300 import binding
    Hd, Wd, insts = _batch(torch)
    n = len(insts)
    with binding.Precoder(max_instances=n, max_M=1024, max_K=256) as prec:
        status = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        prec.precode(insts, status)
        torch.cuda.synchronize()
        ref = [w.cpu().numpy().copy() for w in Wd]
        assert (status.cpu().numpy() == 0).all()
    stream = torch.cuda.current_stream().cuda_stream
    free = []
    outs = [(torch.full((n,), -1, dtype=torch.int32, device="cuda"),
             torch.zeros(n, dtype=torch.float32, device="cuda")) for _ in range(2)]
    torch.cuda.synchronize()
    torch_mem = (torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
    for call in range(2):
        for w in Wd:
            w.fill_(complex(np.nan, np.nan))
        st_call, beta_call = outs[call]
        binding.jacpcg_precode_noalloc(insts, "standard", st_call, None, None, beta_call, stream)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert (st_call.cpu().numpy() == 0).all(), call
        assert (beta_call.cpu().numpy() > 0).all()
        for i, w in enumerate(Wd):
            assert _rel(w.cpu().numpy(), ref[i]) <= TOL_W, (call, i)
    # neither call took memory from torch's allocator; and, as supporting
    # evidence only (other processes share the device's free-memory figure),
    # the device's free memory did not move between the two calls
    assert (torch.cuda.memory_allocated(), torch.cuda.memory_reserved()) == torch_mem
    assert free[0] == free[1]


def test_noalloc_rejects_batches_beyond_its_scratch(torch_gpu):
    torch = torch_gpu
    from paper_2305_13925_gb300 import binding
    H = torch.zeros((256, 1024), dtype=torch.complex64, device="cuda")
    W = torch.zeros_like(H)
    big = [binding.instance(H, W, 1.0, 4) for _ in range(9)]     # 9 x K = 256 needs > 8 MiB
    with pytest.raises(binding.JacpcgError) as e:
        binding.jacpcg_precode_noalloc(big)
    assert e.value.status == binding.JACPCG_ENOMEM
    with pytest.raises(binding.JacpcgError) as e:
        binding.jacpcg_precode_noalloc(big[:1], variant=7)
    assert e.value.status == binding.JACPCG_EINVAL
