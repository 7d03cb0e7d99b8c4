"""GPU Hessian rows (Eq. full_hessian; the subsampled rows of Eq.
sampled_hessian2) against the FP64 oracle's rows (hyper-dual numbers through
the oracle's templated energy, one pass per column), element by element:
max |H - H_ref| <= 1e-5 max |H_ref| per row atom.  Periodic water-like box
(l <= 2, a cell narrower than 2 r_c), periodic FCC cell (l <= 3), an open
cluster through the 128-channel FP16-form model (the rows run the FP32 dual
kernels in every form), and a batch of two clusters whose rows are the
concatenation of each one's rows.  The oracle's cost grows as n^2 C, so the
reference systems are small and the models narrow (32 channels) where the
128-channel width is not the point."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def B():
    import torch
    torch.cuda.init()
    from paper_2605_22698_gb300 import build
    build.build()
    from paper_2605_22698_gb300 import binding
    binding.lib()
    return binding


def _narrow(L):
    return synth.ModelSpec(S=4, T=2, C=32, L=L, H=64, avg_nb=40.0)


def _oracle_rows(om, s, atom):
    return np.stack([om.hessian_row(s.pos, s.species, s.cell, s.pbc, atom, a) for a in range(3)])  # [3][n][3]


def _check(got, ref, label):
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f" {label}: max|dH|/max|H| = {err:.2e} (bar {TOL:g})", end="")
    assert err <= TOL, (label, err)


def test_rows_periodic_water_box(B):
    spec = _narrow(2)
    w = synth.make_weights(spec, 21)
    s = synth.water_box(12, synth.water_side_for(12), seed=7)  # 36 atoms, 7.1 A cell
    om = oracle.Model(spec, w)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    atoms = [0, 25]
    rows = m.hessian_rows([(s.pos, s.species, s.cell, s.pbc)], [atoms])
    assert rows.shape == (2, 3, s.n, 3)
    for k, a in enumerate(atoms):
        _check(rows[k], _oracle_rows(om, s, a), f"water36 atom {a}")
    m.close()


def test_rows_periodic_fcc_l3(B):
    spec = _narrow(3)
    w = synth.make_weights(spec, 31)
    s = synth.fcc((2, 2, 2), seed=3)  # 32 atoms in a 7.2 A cube: several images of each atom
    om = oracle.Model(spec, w)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    rows = m.hessian_rows([(s.pos, s.species, s.cell, s.pbc)], [[9]])
    _check(rows[0], _oracle_rows(om, s, 9), "fcc32 atom 9")
    m.close()


def test_rows_fp16_form_model(B):
    spec = synth.model_spec("water")
    w = synth.make_weights(spec, 21)
    s = synth.cluster(12, seed=5, side=4.5)
    om = oracle.Model(spec, w)
    m = B.Model(spec, w, B.MLIP_PREC_F16)
    rows = m.hessian_rows([(s.pos, s.species, s.cell, s.pbc)], [[4]])
    _check(rows[0], _oracle_rows(om, s, 4), "cluster12 C128 atom 4")
    m.close()


def test_rows_of_a_batch_concatenate_each_systems_rows(B):
    spec = _narrow(2)
    w = synth.make_weights(spec, 4)
    a, b = synth.cluster(14, seed=11, side=5.0), synth.cluster(10, seed=12, side=5.0)
    om = oracle.Model(spec, w)
    m = B.Model(spec, w, B.MLIP_PREC_FP32)
    ra = [[3, 13], [0, 9]]  # row rho: atom ra[g][rho] of system g
    rows = m.hessian_rows([(a.pos, a.species, a.cell, a.pbc), (b.pos, b.species, b.cell, b.pbc)], ra)
    assert rows.shape == (2, 3, a.n + b.n, 3)
    for rho in range(2):
        ref = np.concatenate([_oracle_rows(om, a, ra[0][rho]), _oracle_rows(om, b, ra[1][rho])], axis=1)
        _check(rows[rho], ref, f"batch row {rho}")
    # the second system alone gives its part of the rows bit for bit
    one = m.hessian_rows([(b.pos, b.species, b.cell, b.pbc)], [[0]])
    assert np.array_equal(one[0], rows[0][:, a.n:])
    m.close()


def test_rows_invalid_arguments(B):
    s = synth.cluster(20, seed=3)
    spec = synth.model_spec("water_mace")
    m = B.Model(spec, synth.make_weights(spec, 21), B.MLIP_PREC_FP32)
    with pytest.raises(B.MlipError) as e:  # the symmetric contraction has no GPU rows
        m.hessian_rows([(s.pos, s.species, s.cell, s.pbc)], [[0]])
    assert e.value.code == B.MLIP_ERR_INVALID_ARG
    m.close()
    spec = _narrow(2)
    m = B.Model(spec, synth.make_weights(spec, 21), B.MLIP_PREC_FP32)
    with pytest.raises(B.MlipError) as e:  # a row atom outside its system
        m.hessian_rows([(s.pos, s.species, s.cell, s.pbc)], [[20]])
    assert e.value.code == B.MLIP_ERR_INVALID_ARG
    m.close()
