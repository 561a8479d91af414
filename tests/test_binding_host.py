"""Host-side argument checks of the Python binding, which refuse a call
before the library could read or write past a buffer's end (no GPU needed:
every check runs before the library is called)."""
import numpy as np
import pytest

from paper_1810_05268_gb300 import ckfwi as C

GRID = C.GridSpec(2, (30, 40), 5, 10.0, 4, 1.0, 20, 3.0)
REC = np.array([[10.0, 0.0, 20.0 * i] for i in range(6)])
SHOT = C.ShotSpec(src=(20.0, 0.0, 100.0), rec=REC)


def _dobs(rows=GRID.nt + 1, nrec=6):
    return np.zeros((rows, nrec), np.float32)


def test_short_observed_data_is_refused():
    with pytest.raises(ValueError, match="d_obs"):
        C.adjoint_gradient(None, GRID, SHOT, _dobs(rows=GRID.nt), 4)
    with pytest.raises(ValueError, match="d_obs"):
        C.misfit(None, GRID, SHOT, _dobs(nrec=5))
    with pytest.raises(ValueError, match="d_obs"):
        C.batch_gradient(None, GRID, [SHOT, SHOT], [_dobs(), _dobs(rows=3)], 4)


def test_short_outputs_are_refused():
    with pytest.raises(ValueError, match="grad"):
        C.adjoint_gradient(None, GRID, SHOT, _dobs(), 4, grad=np.zeros(GRID.npts - 1, np.float32))
    with pytest.raises(ValueError, match="d_sim"):
        C.forward_shot(None, GRID, SHOT, d_sim=np.zeros((GRID.nt, 6), np.float32))
    with pytest.raises(ValueError, match="grad_sum"):
        C.batch_gradient(None, GRID, [SHOT], [_dobs()], 4, grad_sum=np.zeros(10))


def test_wrong_dtype_or_layout_is_refused():
    with pytest.raises(ValueError):
        C.adjoint_gradient(None, GRID, SHOT, _dobs().astype(np.float64), 4)
    with pytest.raises(ValueError):
        C.adjoint_gradient(None, GRID, SHOT, np.asfortranarray(np.zeros((GRID.nt + 1, 6, 2), np.float32)), 4)


def test_short_wavelet_is_refused():
    short = C.ShotSpec(src=SHOT.src, rec=REC, wavelet=np.ones(GRID.nt - 1, np.float32))
    with pytest.raises(ValueError, match="wavelet"):
        C.adjoint_gradient(None, GRID, short, _dobs(), 4)
    ok = C.ShotSpec(src=SHOT.src, rec=REC, wavelet=np.ones(GRID.nt, np.float32))
    assert ok.c(GRID.nt).nrec == 6


def test_unknown_storage_mode_is_refused():
    with pytest.raises(ValueError, match="store_mode"):
        C.adjoint_gradient(None, GRID, SHOT, _dobs(), 4, store_mode="fp8")


def test_medium_size_is_checked():
    m = C.Model.__new__(C.Model)
    m.grid, m.h = GRID, None
    with pytest.raises(ValueError, match="medium"):
        m.set_model(np.ones(GRID.npts - 1, np.float32))


def test_names_map_to_the_header_modes():
    o = C._opts(5, "rate", 0.0, 0, C.SLOWNESS2, False, rate=12)
    assert (o.store_mode, o.rate, o.ckpt_slots) == (C.STORE_CODEC_RATE, 12, 5)
    for name, v in C.STORE_NAMES.items():
        assert C._opts(3, name, 1e-3, 0, C.VELOCITY, True).store_mode == v
