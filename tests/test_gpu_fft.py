"""The library's batched complex FFT (mf_fft_c2c: the four-step kernels of the
filter, exposed as the batched transforms the paper timed in Figs. 1-2)
against FP64 references: numpy's pocketfft and the oracle's radix-2 FFT.

Bound: for an FP32 FFT of length N the error of any output is at most about
eps log2(N) ||x||_2 (eps = 2^-24 per butterfly level, errors adding at most
linearly through log2 N levels); the tests allow 7 eps log2(N) ||x||_2 per
transform: |y_gpu - y_ref| <= 4e-7 log2(N) ||x||_2."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0906_4175_gb300 import build
    build.build()
    import paper_0906_4175_gb300 as m
    return m


def _check(y, x64, sign):
    ref = np.fft.fft(x64, axis=-1) if sign < 0 else np.fft.ifft(x64, axis=-1) * x64.shape[-1]
    N = x64.shape[-1]
    tol = 4e-7 * np.log2(N) * np.sqrt(np.sum(np.abs(x64) ** 2, axis=-1, keepdims=True))
    err = np.abs(y.astype(np.complex128) - ref)
    assert np.all(err <= tol), float(np.max(err / tol))


@pytest.mark.parametrize("lg,batch", [(10, 7), (11, 3), (12, 5), (13, 2), (14, 3), (15, 1), (16, 2), (17, 1),
                                      (18, 2), (19, 1), (20, 1), (21, 1), (22, 1)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_numpy(mf, lg, batch, sign):
    import torch
    N = 1 << lg
    rng = np.random.default_rng([lg, batch, sign + 2])
    x = (rng.standard_normal((batch, N)) + 1j * rng.standard_normal((batch, N))).astype(np.complex64)
    y = mf.fft(torch.from_numpy(x).cuda(), sign=sign).cpu().numpy()
    _check(y, x.astype(np.complex128), sign)


@pytest.mark.parametrize("lg,batch", [(10, 131073), (12, 32769)])
def test_fft_in_place_and_large_batch(mf, lg, batch):
    """In place with a ragged batch: N = 2^10 through the single-pass kernel
    (8 sequences per CTA, 131073 of them), N = 2^12 through the four-step
    passes with a batch one larger than an exchange chunk (1 GiB / 8 N)."""
    import torch
    N = 1 << lg
    rng = np.random.default_rng(5 + lg)
    x = (rng.standard_normal((batch, N), dtype=np.float32)
         + 1j * rng.standard_normal((batch, N), dtype=np.float32)).astype(np.complex64)
    t = torch.from_numpy(x).cuda()
    mf.fft(t, sign=-1, out=t)
    y = t.cpu().numpy()
    for b in sorted({0, 1, batch // 2 - 1, batch // 2, batch - 2, batch - 1}):
        _check(y[b:b + 1], x[b:b + 1].astype(np.complex128), -1)


def test_fft_matches_oracle_fft(mf):
    """Same transform as the oracle's own FP64 radix-2 FFT (pinned against the
    direct DFT in the oracle tests)."""
    import torch
    N = 1 << 16
    rng = np.random.default_rng(9)
    x = (rng.standard_normal(N) + 1j * rng.standard_normal(N)).astype(np.complex64)
    y = mf.fft(torch.from_numpy(x[None, :]).cuda(), sign=+1).cpu().numpy()[0]
    ref = oracle.fft(x.astype(np.complex128), +1)
    tol = 4e-7 * 16 * np.sqrt(np.sum(np.abs(x.astype(np.complex128)) ** 2))
    assert np.max(np.abs(y - ref)) <= tol
