"""Host-side input generators (no method arithmetic): layout and the precision-sweep recipe."""
import numpy as np

from paper_2403_10706_b300 import phantom as ph


def test_pairs_are_c_contiguous_float32_with_and_without_noise():
    for pr in (ph.make_pair("tiny"), ph.make_pair("tiny", noise=0.0)):
        for a in (pr.Ip, pr.Im, pr.I_true, pr.b_true):
            assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
        assert pr.b_true.shape == ph.field_dims(pr.dims, pr.pe_dim)


def test_sweep_pairs_share_the_field_and_differ_in_contrast_and_noise():
    a, b = ph.make_sweep_pair(0), ph.make_sweep_pair(1)
    assert a.dims == (144, 168, 111) and a.pe_dim == 1
    assert a.b_true is b.b_true and np.abs(a.b_true).max() <= 8.0 + 1e-6
    for p in (a, b):
        assert p.Ip.flags["C_CONTIGUOUS"] and p.Ip.dtype == np.float32
    # contrast c_i = I_true_i / I_true_base, inside U(0.2, 1)
    base = ph._sweep_base["pair"].I_true
    k = np.unravel_index(np.argmax(base), base.shape)
    ca, cb = a.I_true[k] / base[k], b.I_true[k] / base[k]
    assert 0.2 <= ca <= 1.0 and 0.2 <= cb <= 1.0 and abs(ca - cb) > 1e-6
    # noise of standard deviation 0.03 on top of the scaled noise-free pair
    resid = a.Ip.astype(np.float64) - ca * ph._sweep_base["pair"].Ip
    assert abs(resid.std() - 0.03) < 1e-3
    np.testing.assert_array_equal(ph.make_sweep_pair(0).Ip, a.Ip)   # seeded
