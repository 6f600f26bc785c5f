"""The identity behind the folded forward plane pass, checked with numpy's FFT
(no GPU): the output rows y = F k + h of the 2D inverse DFT of an NY x NX
plane a are the (NY/F)-point inverse DFT along y, and the NX-point one along
x, of the folded rows

    b_h[r] = W^{h r} sum_{q < F} a[r + (NY/F) q] (W^{NY/F})^{h q},   r < NY/F,

with W = exp(2 pi i / NY) (unnormalised transforms). The GPU kernel runs this
with F = 4 on 256^2 planes and F = 2 on 128^2 planes; its results are checked
against the oracle in the GPU parity tests."""
import numpy as np
import pytest


def _idft2(a):
    return np.fft.ifft2(a) * a.size


@pytest.mark.parametrize("ny,nx,F", [(128, 128, 2), (256, 256, 4), (128, 160, 2), (64, 32, 4)])
def test_output_rows_mod_f_are_transforms_of_the_folded_rows(ny, nx, F):
    rng = np.random.default_rng(ny + nx + F)
    a = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    full = _idft2(a)
    nh = ny // F
    W = np.exp(2j * np.pi / ny)
    r = np.arange(nh)[:, None]
    for h in range(F):
        b = sum(a[q * nh:(q + 1) * nh] * W ** (nh * h * q) for q in range(F)) * W ** (h * r)
        assert np.allclose(_idft2(b), full[h::F], rtol=0, atol=1e-9 * np.abs(full).max())


def test_fold_is_not_the_plain_sum():
    """Dropping the row factor W^{h r} (a plausible mistake) breaks the identity."""
    rng = np.random.default_rng(5)
    a = rng.standard_normal((16, 8)) + 1j * rng.standard_normal((16, 8))
    full = _idft2(a)
    b = a[:8] - a[8:]          # h = 1 of F = 2 without W^{r}
    assert not np.allclose(_idft2(b), full[1::2])
