"""The device noise generator against the oracle, through the C ABI.

* Raw Philox4x32-10 blocks, bit for bit, over 2^20 + 7 counters in several
  counter families (sample noise of plain and proposal streams, a large
  race tag, the prediction-perturbation word), computed by the same
  round-key form the sample loop uses; the device also checks that form
  against the key-schedule form of the winner re-roll (no mismatch).
* The FP32 Box-Muller normals of the sample loop against the oracle's FP64
  normals of the same words: |dz| <= 2e-5 (1 + |z|), the accuracy of the
  hardware logarithm, square root, sine and cosine approximations.
* The FP32 FMA probe runs and reports a plausible rate.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _L():
    from paper_2607_25388_b300 import _lib
    return _lib.lib()


def _vp(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("seed,c1,c2,c3", [
    (0x0123456789ABCDEF, 0, 3 | (1 << 16), 0),                   # sample noise, step pair 0, vehicle 3, round 1
    (7, 29 | (1 << 31), 9 | (6 << 16), 1255),                     # proposal stream, extra round, batch race
    (2**64 - 1, 63, 15 | (4095 << 16), 2**31 - 1),                 # extreme words
    (200, 0, 2 | (3 << 16), 0),
])
def test_philox_words_bit_exact(seed, c1, c2, c3):
    L = _L()
    n = (1 << 20) + 7
    k0 = 0xFFFFF000 if c3 == 2**31 - 1 else 0                       # wrap of the k word
    words = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    mism = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = L.sgtp_philox_words(seed, c1, c2, c3, k0, n, _vp(words), _vp(mism), None)
    assert st == 0, L.sgtp_last_error()
    torch.cuda.synchronize()
    dev = words.cpu().numpy().view(np.uint32)
    ref = O.philox_batch(c1, c2, c3, k0, n, seed)
    bad = np.nonzero(np.any(dev != ref, axis=1))[0]
    assert bad.size == 0, f"{bad.size} blocks differ, first at i={bad[:5]}"
    assert int(mism.item()) == 0


def test_sample_normals_match_oracle():
    L = _L()
    seed, race, agent, rnd = 12345, 17, 4, 2
    nk, T = 4096, 61                                                # odd T: the last pair's second half unused
    for stream in (0, 1):
        z = torch.empty((nk, T, 2), dtype=torch.float32, device="cuda")
        st = L.sgtp_noise_normals(seed, race, agent, rnd, stream, 1000, nk, T, _vp(z), None)
        assert st == 0, L.sgtp_last_error()
        torch.cuda.synchronize()
        zg = z.cpu().numpy().astype(np.float64)
        zo = O.std_normals_batch(seed, race, agent, rnd, stream, 1000, nk, T)
        err = np.abs(zg - zo) / (1.0 + np.abs(zo))
        assert err.max() <= 2e-5, f"stream {stream}: worst {err.max():.2e}"
        # moments of 0.5 M draws: mean 0, variance 1
        assert abs(zg.mean()) < 0.01 and abs(zg.var() - 1.0) < 0.01


def test_fma_probe_reports_a_plausible_rate():
    from paper_2607_25388_b300 import roofline as R
    tf, form = R.measure_fma_peak(reps=2, iters=4000)
    nominal = R.fp32_peak_tflops(sms=torch.cuda.get_device_properties(0).multi_processor_count)
    assert 0.3 * nominal < tf < 1.3 * nominal, (tf, form, nominal)


def test_fma_probe_rejects_bad_arguments():
    L = _L()
    sink = torch.zeros(8, device="cuda")
    n0 = L.sgtp_launch_count()
    fl = C.c_double()
    assert L.sgtp_fma_probe(0, 10, 0, _vp(sink), None, C.byref(fl)) == 1
    assert L.sgtp_fma_probe(1, 0, 0, _vp(sink), None, C.byref(fl)) == 1
    assert L.sgtp_launch_count() == n0
