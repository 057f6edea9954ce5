"""Host arithmetic of bench.py, pinned on CPU: the algorithmic flop counts
against the Appendix's operation counts (oracle module) and brute-force MAC
counts, the algorithmic bytes against the tensors the path must move, and the
oracle baseline's one-thread figure."""
import numpy as np

import bench
from oracle import oracle as O


def _brute_gram_macs(M, K):
    # complex MACs of the lower triangle (i >= j) of H^H H: M per entry
    return sum(M for i in range(K) for j in range(i + 1))


def test_flops_per_instance():
    for M, K, T in ((16, 3, 2), (100, 32, 5), (1024, 64, 6)):
        f = bench.flops_per_instance(M, K, T)
        assert f["gram"] == 8 * _brute_gram_macs(M, K)          # 8 real flops per complex MAC
        assert f["hx"] == 8 * M * K * K                          # W = H X: M K K MACs
        # K right-hand sides, T iterations each (Appendix), Jacobi preprocessing once per matrix
        assert f["pcg"] == K * O.flops_cg(K, T) + O.flops_jacobi_preprocessing(K)


def test_algorithmic_bytes():
    for M, K in ((16, 3), (1024, 64), (4096, 256)):
        h = np.zeros((M, K), dtype=np.complex64).nbytes
        a = np.zeros((K, K), dtype=np.complex64).nbytes
        assert bench.algorithmic_bytes("gram", M, K) == h + a      # read H, write A
        assert bench.algorithmic_bytes("hx", M, K) == 2 * h + a    # read H and X, write W


def test_cpu_baseline_one_core():
    from paper_2305_13925_gb300 import channels as C
    H, xi = C.generate_batch("single_256x16", 6, 0)
    Hst = np.ascontiguousarray(np.swapaxes(H, 1, 2)).astype(np.complex64)
    out, acc = bench.cpu_baseline_leg(Hst, xi, 8, "standard", 0.2)
    assert acc is None
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] >= 1
    one = out["one_core"]
    assert one["cores"] == 1 and one["value"] > 0 and one["unit"] == out["unit"]
