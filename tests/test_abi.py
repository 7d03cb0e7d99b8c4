"""Host-side checks of the C ABI library (no GPU needed): it builds for
sm_103a, loads, exports every function include/mlip.h declares, and its
host-only entry points answer without touching a device."""
import ctypes

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def lib():
    from paper_2605_22698_gb300 import build
    build.build()
    from paper_2605_22698_gb300 import binding
    return binding


def test_exports_every_declared_symbol(lib):
    names = lib.exported_symbols()
    assert "mlip_energy_forces" in names and "mlip_neighbors" in names
    L = lib.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_num_weights_matches_generator(lib):
    for name in ("small", "water", "fcc"):
        spec = synth.model_spec(name)
        assert lib.mlip_model_num_weights(lib.make_desc(spec)) == spec.n_weights()


def test_num_weights_rejects_bad_hyperparameters(lib):
    spec = synth.model_spec("water")
    d = lib.make_desc(spec)
    d.l_max = 5
    with pytest.raises(lib.MlipError) as e:
        lib.mlip_model_num_weights(d)
    assert e.value.code == lib.MLIP_ERR_INVALID_ARG
    assert b"l_max" in lib.lib().mlip_last_error()


def test_params_file_roundtrip_layout(tmp_path):
    spec = synth.model_spec("small")
    w = synth.make_weights(spec, 1)
    p = tmp_path / "m.bin"
    synth.write_params(str(p), spec, w)
    raw = p.read_bytes()
    assert raw[:8] == b"MLIPPRM1"
    tail = np.frombuffer(raw[-4 * w.size:], dtype="<f4")
    np.testing.assert_array_equal(tail, w)
