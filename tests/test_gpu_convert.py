"""The precision form's FP32 <-> FP64 conversions on the integer pipes
(hrm_probe_convert) against the hardware conversions, bit for bit.

The precision-form kernels convert many values per cell and per midpoint and
build the converted encodings with integer operations (FP64-pipe instructions
are scarce on GB300). They must give exactly what a hardware conversion gives:
round to nearest with ties to even for FP64 -> FP32, exact widening for
FP32 -> FP64, over every exponent range, zeros, subnormals, overflow,
infinities and NaN.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_04488_gb300 import build
    build.build()
    from paper_2208_04488_gb300 import hrm as H
    return H


def _doubles(rng, n):
    bits = rng.integers(0, 2**63, size=n, dtype=np.int64).view(np.uint64)
    bits[: n // 4] ^= np.uint64(1) << np.uint64(63)
    uniform_bits = bits.view(np.float64)  # every exponent, NaN and infinities
    mag = 10.0 ** rng.uniform(-46, 39, size=n)  # around the float range and its edges
    signed = np.where(rng.random(n) < 0.5, -mag, mag)
    f = rng.standard_normal(n).astype(np.float32) * np.float32(1e3)
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    ties = f.astype(np.float64) + 0.5 * ulp  # exact halfway cases, both parities
    near = np.concatenate([ties, np.nextafter(ties, np.inf), np.nextafter(ties, -np.inf)])
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    edges = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, np.nextafter(fmax, np.inf),
                      fmax + 2.0 ** 103, 2.0 ** 128, tiny, -tiny,  # fmax + half its ulp: the tie that rounds to infinity
                      np.nextafter(tiny, 0.0), tiny * (1 - 2.0 ** -25), tiny * 0.5, 1e-45, 5e-324, 1.0, -1.0,
                      1.0 - 2.0 ** -25, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24])
    return np.concatenate([uniform_bits, signed, near, edges])


def _floats(rng, n):
    bits = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    edges = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.1754942e-38, 1.17549435e-38,
                      3.4028235e38, -3.4028235e38, 1.0, -2.5], dtype=np.float32)
    return np.concatenate([bits.view(np.float32), edges])


def test_integer_conversions_match_the_hardware(hrm):
    import torch
    rng = np.random.default_rng(2024)
    d = _doubles(rng, 200000)
    f = _floats(rng, d.size)[: d.size]
    if f.size < d.size:
        f = np.resize(f, d.size)
    td = torch.from_numpy(d).cuda()
    tf = torch.from_numpy(f).cuda()
    narrowed, widened = hrm.probe_convert(td, tf)
    torch.cuda.synchronize()
    ref_n = td.float()
    ref_w = tf.double()
    nb, rb = narrowed.view(torch.int32), ref_n.view(torch.int32)
    wb, rw = widened.view(torch.int64), ref_w.view(torch.int64)
    bad_n = (nb != rb) & ~(torch.isnan(narrowed) & torch.isnan(ref_n))
    bad_w = (wb != rw) & ~(torch.isnan(widened) & torch.isnan(ref_w))
    assert int(bad_n.sum()) == 0, d[bad_n.cpu().numpy()][:5]
    assert int(bad_w.sum()) == 0, f[bad_w.cpu().numpy()][:5]
