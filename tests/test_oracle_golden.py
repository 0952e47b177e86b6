"""Oracle thresholding stages against hand-worked fixtures (tests/golden/)."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.golden_io import load

CASES = ["rfi_3x8_channel.txt", "rfi_3x8_spectrum.txt", "rfi_8x64_float.txt", "rfi_4x16_spectrum_unflagged.txt"]


def _x(g, dtype):
    if dtype == "u8":
        return g["x"].astype(np.uint8)
    return g["x"].astype(np.float32)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("as_float", [False, True])
@pytest.mark.parametrize("dil", [False, True])
def test_golden_rfi(name, as_float, dil):
    g = load(name)
    dtype = g["meta"]["dtype"]
    if as_float:
        dtype = "f32"
    x = _x(g, dtype)
    rfi = O.RfiParams(chunk_width=int(g["meta"]["W"]), tau_channel=float(g["meta"]["tau_channel"]),
                      tau_spectrum=float(g["meta"]["tau_spectrum"]), dilate_channels=dil)
    st = O.bandpass(x, dtype)
    raw, flag = O.channel_mask(x, dtype, st, rfi)
    spec = O.spectrum_mask(x, dtype, st, rfi, flag)
    assert np.array_equal(raw, g["raw"].astype(np.uint8))
    want = g["flag_dilate_channels"] if dil else g["flag"]
    assert np.array_equal(flag, want.astype(np.uint8))
    assert np.array_equal(spec, g["spec"].astype(np.uint8))
