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
    for name in ("small", "water", "fcc", "small_mace", "water_mace", "fcc_mace", "small_charged", "water_charged",
                 "water_mace_charged", "water_gated", "fcc_gated", "water_mace_gated"):
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


_LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "mlip.h"
#define F(T, m) printf(#T " " #m " %zu\n", offsetof(T, m));
#define Z(T) printf(#T " sizeof %zu\n", sizeof(T));
int main(void) {
  F(mlip_model_desc, cutoff) F(mlip_model_desc, masses) F(mlip_model_desc, correlation)
  F(mlip_model_desc, charges) F(mlip_model_desc, coulomb_r0) F(mlip_model_desc, gate) F(mlip_model_desc, parity)
  Z(mlip_model_desc)
  F(mlip_serve_config, max_slots) F(mlip_serve_config, bucket_edges) F(mlip_serve_config, device_poll_limit_us)
  F(mlip_serve_config, resident_after)
  Z(mlip_serve_config)
  F(mlip_request, n) F(mlip_request, pos) F(mlip_request, cell) F(mlip_request, pbc) F(mlip_request, vel)
  F(mlip_request, seed) F(mlip_request, dt_fs) Z(mlip_request)
  F(mlip_result, energy) F(mlip_result, stress) F(mlip_result, forces) F(mlip_result, ke) F(mlip_result, t_done)
  Z(mlip_result)
  F(mlip_serve_statistics, elapsed_s) F(mlip_serve_statistics, device_bytes) F(mlip_serve_statistics, n_buckets)
  F(mlip_serve_statistics, bucket_count) F(mlip_serve_statistics, bucket_p99_ms) F(mlip_serve_statistics, skin_steps)
  F(mlip_serve_statistics, skin_builds) F(mlip_serve_statistics, changed_iterations)
  F(mlip_serve_statistics, changed_busy_s) Z(mlip_serve_statistics)
  F(mlip_md_options, rebuild_every) F(mlip_md_options, use_graph) Z(mlip_md_options)
  F(mlip_md_report, redone_blocks) F(mlip_md_report, max_candidates) F(mlip_md_report, max_displacement)
  Z(mlip_md_report)
  return 0;
}
"""


def test_struct_layouts_match_the_header(lib, tmp_path):
    """The binding's ctypes structures have the C header's offsets and sizes."""
    import os
    import subprocess
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    for line in out.strip().splitlines():
        tname, field, val = line.split()
        T = getattr(lib, tname)
        got = ctypes.sizeof(T) if field == "sizeof" else getattr(T, field).offset
        assert got == int(val), (tname, field, got, val)


def test_params_file_version_2_header(tmp_path):
    """Models with the contraction, the charge head or the gate are written as
    version 2: after the 8 hyperparameters, i32 correlation, i32 charges,
    f64 coulomb_r0, i32 gate, then rc and avg_nb as in version 1."""
    import struct
    spec = synth.model_spec("water_mace_charged")
    import dataclasses
    spec = dataclasses.replace(spec, gate=1)
    w = synth.make_weights(spec, 2)
    p = tmp_path / "v2.bin"
    synth.write_params(str(p), spec, w)
    raw = p.read_bytes()
    assert raw[:8] == b"MLIPPRM1" and struct.unpack_from("<I", raw, 8)[0] == 2
    assert list(struct.unpack_from("<8i", raw, 12)) == list(spec.hyper)
    corr, charges, r0, gate = struct.unpack_from("<iidi", raw, 44)
    assert (corr, charges, r0, gate) == (2, 1, 2.5, 1)
    rc, avg = struct.unpack_from("<2d", raw, 64)
    assert (rc, avg) == (spec.rc, spec.avg_nb)
    assert struct.unpack_from("<q", raw, 80 + 8 * spec.S)[0] == w.size == spec.n_weights()
    # version 1 for the plain model
    plain = synth.model_spec("small")
    q = tmp_path / "v1.bin"
    synth.write_params(str(q), plain, synth.make_weights(plain, 1))
    assert struct.unpack_from("<I", q.read_bytes(), 8)[0] == 1
