"""Seeded synthetic XL-MIMO channels (input generation only).

This module produces the channel matrices H that both the CUDA path and the
FP64 oracle consume.  It holds none of the precoder's arithmetic (no Gram
matrix, no iteration, no precoder): only the channel model of Sec. II,
Eqs. 2-4, and the workload shapes the library is measured on.

Channel model (Sec. II, Eqs. 2-4).  The M antennas form S subarrays of
M_s = M/S antennas.  For user k and subarray s,

    h_{s,k} = sqrt(beta_{s,k}) * R_s^{1/2} g_{s,k},   g ~ CN(0, I)

when subarray s lies in user k's visibility region (VR), and h_{s,k} = 0
otherwise (the indicator D_k of Eq. 4).  R_s is the exponential correlation
matrix R_s[i, j] = r_s^{|i-j|}.  Any square root of R_s gives the same
distribution; we apply its lower Cholesky factor, which for this matrix is
the first-order autoregression y_0 = g_0, y_i = r y_{i-1} + sqrt(1-r^2) g_i
(covariance r^{|i-j|}, unit variance).  beta_{s,k} is log-normal shadowing:
10 log10(beta) ~ N(mean_db, sigma_db^2), normalised to a noise floor at
mean_db, so the noise variance is 1 and the transmit power equals the SNR.
The VR of a user is a contiguous run of n_vis subarrays whose first
subarray is uniform over the admissible starts.

The paper's own geometric preset (Table I: ULA, spacing 2 lambda at
2.6 GHz, path loss Omega d^{-nu} per antenna, VR centre U(0, N) and length
LN(0.1 N, 0.1)) is available as ``paper_table1``.

Randomness.  Every random number comes from a counter-based generator:
SplitMix64's output function (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to
key + (index + 1) * 0x9E3779B97F4A7C15, where the key hashes
(seed, stream, instance).  Uniforms are (z >> 11 + 0.5) * 2^-53 in (0, 1);
normals come from the Box-Muller transform.  A channel therefore depends
only on (seed, instance index, preset), not on batch composition or order.

Storage.  ``H`` arrays are returned in math shape (n, M, K) complex128
holding values already rounded to the input precision (complex64, or
bfloat16 per real component), so that an exact upcast feeds the oracle the
very numbers the GPU reads.  ``to_device_layout`` gives the column-major,
interleaved (re, im) layout of the C-ABI.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (kept apart so that streams never share counters)
_STREAM_PARAMS = 1
_STREAM_SHADOW = 2
_STREAM_SMALL = 3
_STREAM_SIZE = 4
_STREAM_GEOM = 5


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=False)
    z = (z ^ (z >> np.uint64(30))) * _C1
    z = (z ^ (z >> np.uint64(27))) * _C2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int, inst: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        k = _mix64(np.array([k ^ np.uint64(stream) * _GAMMA], dtype=np.uint64))[0]
        k = _mix64(np.array([k ^ np.uint64(inst & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64))[0]
    return np.uint64(k)


def uniform(seed: int, stream: int, inst: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in (0, 1) at counters ``idx`` of (seed, stream, inst)."""
    key = _key(seed, stream, inst)
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(key + (idx + np.uint64(1)) * _GAMMA)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal_pair(seed: int, stream: int, inst: int, idx: np.ndarray):
    """Two independent N(0,1) arrays from counters 2*idx and 2*idx+1 (Box-Muller)."""
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = uniform(seed, stream, inst, idx * np.uint64(2))
    u2 = uniform(seed, stream, inst, idx * np.uint64(2) + np.uint64(1))
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)


@dataclasses.dataclass(frozen=True)
class ChannelSpec:
    """Shape and statistics of one family of synthetic instances."""

    M: int
    S: int
    K: int
    r: tuple                       # (lo, hi) of the per-subarray correlation, lo == hi for fixed
    n_vis: tuple                   # (lo, hi) visible subarrays per user, contiguous
    snr_db: tuple                  # SNR choices in dB, one drawn uniformly per instance
    shadow_mean_db: float = -100.0
    shadow_sigma_db: float = 8.0
    xi_rule: str = "K/SNR"         # regulariser: "K/SNR" or "1/SNR" (Sec. II after Eq. 7)

    @property
    def Ms(self) -> int:
        return self.M // self.S


PRESETS = {
    # M=256 as 4 subarrays of 64, K=16, r=0.5, 2 of 4 subarrays visible, SNR 10 dB
    "single_256x16": ChannelSpec(M=256, S=4, K=16, r=(0.5, 0.5), n_vis=(2, 2), snr_db=(10.0,)),
    # M=1024 as 8 subarrays of 128, K=64, r ~ U[0.3, 0.9], 2..6 of 8 visible, SNR in {0, 10, 20}
    "batched_1024x64": ChannelSpec(M=1024, S=8, K=64, r=(0.3, 0.9), n_vis=(2, 6),
                                   snr_db=(0.0, 10.0, 20.0)),
    # M=4096 as 16 subarrays of 256, K=256, 4..12 of 16 visible
    "xl_4096x256": ChannelSpec(M=4096, S=16, K=256, r=(0.3, 0.9), n_vis=(4, 12),
                               snr_db=(0.0, 10.0, 20.0)),
}

# ragged mix: K and M drawn per instance from these sets, S = 8, 2..6 visible
RAGGED_K = (8, 16, 32, 64, 128, 256)
RAGGED_M = (256, 512, 1024, 2048, 4096)


@dataclasses.dataclass
class Instance:
    """One synthetic channel: H in math shape (M, K) and its regulariser."""

    H: np.ndarray          # complex128 (M, K), values exactly representable in the input dtype
    xi: float
    snr_db: float
    spec: ChannelSpec


def _ar1_columns(g: np.ndarray, r: float) -> np.ndarray:
    """Apply the lower Cholesky factor of R[i,j] = r^{|i-j|} along axis 0."""
    y = np.empty_like(g)
    y[0] = g[0]
    c = math.sqrt(max(0.0, 1.0 - r * r))
    for i in range(1, g.shape[0]):
        y[i] = r * y[i - 1] + c * g[i]
    return y


def round_complex64(H: np.ndarray) -> np.ndarray:
    """Round to complex64 and upcast exactly back to complex128."""
    return H.astype(np.complex64).astype(np.complex128)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even), as float32."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).reshape(f.shape)


def round_complex_bf16(H: np.ndarray) -> np.ndarray:
    """Round each real component to bfloat16 and upcast exactly to complex128."""
    re = round_bf16(H.real.astype(np.float32)).astype(np.float64)
    im = round_bf16(H.imag.astype(np.float32)).astype(np.float64)
    return re + 1j * im


def generate_instance(spec: ChannelSpec, seed: int, inst: int, dtype: str = "complex64") -> Instance:
    """Channel ``inst`` of family ``spec`` for ``seed`` (independent of any batch)."""
    M, S, K, Ms = spec.M, spec.S, spec.K, spec.Ms
    assert M % S == 0
    # per-instance parameters: SNR choice, r per subarray, n_vis and start per user
    n_par = 1 + S + 2 * K
    u = uniform(seed, _STREAM_PARAMS, inst, np.arange(n_par))
    snr_db = spec.snr_db[min(int(u[0] * len(spec.snr_db)), len(spec.snr_db) - 1)]
    r_lo, r_hi = spec.r
    r = r_lo + (r_hi - r_lo) * u[1:1 + S]
    v_lo, v_hi = spec.n_vis
    n_vis = v_lo + np.minimum((u[1 + S:1 + S + K] * (v_hi - v_lo + 1)).astype(np.int64), v_hi - v_lo)
    u_start = u[1 + S + K:1 + S + 2 * K]
    start = np.minimum((u_start * (S - n_vis + 1)).astype(np.int64), S - n_vis)
    # shadowing per (user, subarray), normalised to the noise floor
    z, _ = normal_pair(seed, _STREAM_SHADOW, inst, np.arange(K * S))
    gain_db = spec.shadow_sigma_db * z.reshape(K, S)           # (x - mean_db), x ~ N(mean_db, sigma^2)
    amp = np.sqrt(10.0 ** (gain_db / 10.0))
    # small-scale fading g_{k,m} ~ CN(0,1), counter (k*M + m)
    n1, n2 = normal_pair(seed, _STREAM_SMALL, inst, np.arange(K * M))
    g = ((n1 + 1j * n2) / math.sqrt(2.0)).reshape(K, M).T      # (M, K)
    H = np.zeros((M, K), dtype=np.complex128)
    for s in range(S):
        rows = slice(s * Ms, (s + 1) * Ms)
        vis = (start <= s) & (s < start + n_vis)
        if not vis.any():
            continue
        y = _ar1_columns(g[rows][:, vis], float(r[s]))
        H[rows, vis] = y * amp[vis, s][None, :]
    snr_lin = 10.0 ** (snr_db / 10.0)
    xi = (K / snr_lin) if spec.xi_rule == "K/SNR" else (1.0 / snr_lin)
    if dtype == "complex64":
        H = round_complex64(H)
    elif dtype == "bf16":
        H = round_complex_bf16(H)
    elif dtype != "complex128":
        raise ValueError(dtype)
    return Instance(H=H, xi=float(xi), snr_db=float(snr_db), spec=spec)


def generate_batch(preset: str | ChannelSpec, n: int, seed: int, first: int = 0,
                   dtype: str = "complex64"):
    """Uniform batch: H (n, M, K) complex128 and xi (n,) for instances first..first+n-1."""
    spec = PRESETS[preset] if isinstance(preset, str) else preset
    H = np.empty((n, spec.M, spec.K), dtype=np.complex128)
    xi = np.empty(n, dtype=np.float64)
    for i in range(n):
        inst = generate_instance(spec, seed, first + i, dtype)
        H[i] = inst.H
        xi[i] = inst.xi
    return H, xi


def ragged_spec(seed: int, inst: int) -> ChannelSpec:
    """Size of ragged instance ``inst``: K and M uniform over RAGGED_K and RAGGED_M."""
    u = uniform(seed, _STREAM_SIZE, inst, np.arange(2))
    K = RAGGED_K[min(int(u[0] * len(RAGGED_K)), len(RAGGED_K) - 1)]
    M = RAGGED_M[min(int(u[1] * len(RAGGED_M)), len(RAGGED_M) - 1)]
    return ChannelSpec(M=M, S=8, K=K, r=(0.3, 0.9), n_vis=(2, 6), snr_db=(0.0, 10.0, 20.0))


def _ragged_chunk(args):
    seed, a, b, dtype, k_set, m_set = args
    return generate_ragged(b - a, seed, a, dtype, k_set, m_set, workers=1)


def generate_ragged(n: int, seed: int, first: int = 0, dtype: str = "complex64",
                    k_set: Sequence[int] | None = None, m_set: Sequence[int] | None = None,
                    workers: int | None = 1):
    """Ragged batch: list of Instance with per-instance (M, K).  workers > 1
    (or None for the core count) generates in spawned processes (call before
    any GPU work); the result does not depend on the worker count."""
    import os
    if workers is None:
        workers = min(16, os.cpu_count() or 1)
    if workers > 1 and n >= 16:
        import concurrent.futures as cf
        import multiprocessing as mp
        chunks = [(seed, first + i * n // (4 * workers), first + (i + 1) * n // (4 * workers), dtype,
                   k_set, m_set) for i in range(4 * workers)]
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_ragged_chunk, [c for c in chunks if c[2] > c[1]]))
        return [inst for part in parts for inst in part]
    out = []
    for i in range(n):
        spec = ragged_spec(seed, first + i)
        if k_set is not None or m_set is not None:
            u = uniform(seed, _STREAM_SIZE, first + i, np.arange(2))
            ks = tuple(k_set) if k_set is not None else RAGGED_K
            ms = tuple(m_set) if m_set is not None else RAGGED_M
            spec = dataclasses.replace(spec, K=ks[min(int(u[0] * len(ks)), len(ks) - 1)],
                                       M=ms[min(int(u[1] * len(ms)), len(ms) - 1)])
        out.append(generate_instance(spec, seed, first + i, dtype))
    return out


def paper_table1(seed: int, inst: int, M: int = 100, K: int = 32, S: int = 4,
                 snr_db: float = 10.0, r: float = 0.5) -> Instance:
    """Geometric preset after Table I and Sec. IV (oracle tests only).

    ULA of M antennas at spacing 2 lambda, f_c = 2.6 GHz (N = M * 2 lambda);
    users uniform in a 100 m x 100 m square at least 30 m from the array
    centre; per-antenna path loss w = Omega d^{-nu} with Omega = 4, nu = 3
    (Eq. 3); VR centre c_k ~ U(0, N) and length l_k with ln l_k ~ N(ln(0.1 N),
    0.1^2); exponential correlation r inside each subarray (the paper gives
    no correlation model).  Gains are divided by the noise power
    (-50 dBm) so that the noise variance is 1; xi = 1/SNR.
    """
    lam = 299792458.0 / 2.6e9
    d_ant = 2.0 * lam
    N = M * d_ant
    assert M % S == 0
    Ms = M // S
    ant_x = (np.arange(M) + 0.5) * d_ant
    ug = uniform(seed, _STREAM_GEOM, inst, np.arange(64 * K))
    pos = np.empty((K, 2))
    j = 0
    for k in range(K):
        while True:      # rejection sampling for the 30 m exclusion zone around the array centre
            x = ug[j] * 100.0 - 50.0 + N / 2.0
            y = ug[j + 1] * 100.0
            j += 2
            if math.hypot(x - N / 2.0, y) >= 30.0:
                break
        pos[k] = (x, y)
    d = np.sqrt((ant_x[:, None] - pos[None, :, 0]) ** 2 + pos[None, :, 1] ** 2)   # (M, K)
    noise_w = 10.0 ** (-50.0 / 10.0) * 1e-3
    w = 4.0 * d ** (-3.0) / noise_w
    uv = uniform(seed, _STREAM_PARAMS, inst, np.arange(2 * K))
    zv, _ = normal_pair(seed, _STREAM_SHADOW, inst, np.arange(K))
    centre = uv[:K] * N
    length = np.exp(math.log(0.1 * N) + 0.1 * zv)
    vis = np.abs(ant_x[:, None] - centre[None, :]) <= length[None, :] / 2.0
    n1, n2 = normal_pair(seed, _STREAM_SMALL, inst, np.arange(K * M))
    g = ((n1 + 1j * n2) / math.sqrt(2.0)).reshape(K, M).T
    hbar = np.empty_like(g)
    for s in range(S):
        rows = slice(s * Ms, (s + 1) * Ms)
        hbar[rows] = _ar1_columns(g[rows], r)
    H = round_complex64(np.sqrt(w) * vis * hbar)
    spec = ChannelSpec(M=M, S=S, K=K, r=(r, r), n_vis=(0, 0), snr_db=(snr_db,), xi_rule="1/SNR")
    return Instance(H=H, xi=10.0 ** (-snr_db / 10.0), snr_db=snr_db, spec=spec)


def to_device_layout(H: np.ndarray, dtype=np.complex64) -> np.ndarray:
    """(n, M, K) or (M, K) math shape -> per-instance column-major storage.

    Returns an array of shape (n, K, M) (or (K, M)) whose memory is, per
    instance, column k of H contiguous, complex values interleaved (re, im).
    """
    return np.ascontiguousarray(np.swapaxes(H, -1, -2)).astype(dtype)


def to_planar_bf16(H: np.ndarray) -> np.ndarray:
    """(M, K) complex -> (2, K, M) float32 planes (Re, Im) holding bf16-exact values."""
    Hc = np.ascontiguousarray(np.swapaxes(H, -1, -2))
    return np.stack([round_bf16(Hc.real.astype(np.float32)), round_bf16(Hc.imag.astype(np.float32))])


def _fill_device_layout(args):
    """Worker: instances [a, b) of a uniform batch into a shared (n, K, M) complex64 array."""
    from multiprocessing import shared_memory
    name, shape, preset, seed, first, a, b, dtype = args
    shm = shared_memory.SharedMemory(name=name)
    try:
        out = np.ndarray(shape, dtype=np.complex64, buffer=shm.buf)
        xi = np.empty(b - a)
        spec = PRESETS[preset] if isinstance(preset, str) else preset
        for i in range(a, b):
            inst = generate_instance(spec, seed, first + i, dtype)
            out[i] = inst.H.T.astype(np.complex64)
            xi[i - a] = inst.xi
        return a, xi
    finally:
        shm.close()


def generate_batch_device_layout(preset: str | ChannelSpec, n: int, seed: int, first: int = 0,
                                 workers: int | None = None, dtype: str = "complex64"):
    """Uniform batch straight into the C-ABI storage layout: returns
    (H (n, K, M) complex64, xi (n,)).  Same values as ``generate_batch``;
    uses a pool of spawned worker processes (call before any GPU work)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    from multiprocessing import shared_memory
    spec = PRESETS[preset] if isinstance(preset, str) else preset
    shape = (n, spec.K, spec.M)
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1 or n < 8:
        H, xi = generate_batch(spec, n, seed, first, dtype)
        return to_device_layout(H), xi
    nbytes = int(np.prod(shape)) * 8
    shm = shared_memory.SharedMemory(create=True, size=nbytes)
    try:
        chunks = [(i * n // (4 * workers), (i + 1) * n // (4 * workers)) for i in range(4 * workers)]
        xi = np.empty(n)
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            jobs = [(shm.name, shape, preset, seed, first, a, b, dtype) for a, b in chunks if b > a]
            for a, x in ex.map(_fill_device_layout, jobs):
                xi[a:a + len(x)] = x
        H = np.ndarray(shape, dtype=np.complex64, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()
    return H, xi
