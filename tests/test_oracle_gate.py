"""Pins of the oracle's gated update with a species-dependent self-connection
(NequIP's gate nonlinearity and self-connection, on this layer's uniform
natural-parity irreps):

    pre_l = m_l W_l + h_l Wself[z][l]              l = 0..L
    g_l   = m_0 Wgate_l + h_0 Wselfgate[z]_l       l = 1..L (one gate per channel)
    h_0  += silu(pre_0),   h_l += sigmoid(g_l) pre_l

Fixed by the definition: with the gate and self-connection weights zero the
gate is 1/2 everywhere, so the model equals the ungated one with its l > 0
mixes doubled; an isolated atom (no messages) reduces to the self-connection
chain on its embedding, computed here by hand.  The whole-model pins
(invariances, forces = dual numbers = differences, stress) run on gated
models in test_oracle_model.py.
"""
import numpy as np

import oracle
import synth


def _split_set(spec, w, name, value):
    w = w.copy()
    off = 0
    for nm, shape, _ in spec.weight_shapes():
        k = int(np.prod(shape))
        if nm == name:
            w[off:off + k] = np.asarray(value, np.float32).reshape(-1)
        off += k
    return w


def test_zero_gate_weights_halve_the_vector_updates():
    base = synth.ModelSpec(S=4, T=2, C=8, L=2, H=16, avg_nb=10.0)
    gated = synth.ModelSpec(S=4, T=2, C=8, L=2, H=16, avg_nb=10.0, gate=1)
    wb = synth.make_weights(base, 17)
    Pb = synth.split_weights(base, wb)
    wg = np.zeros(gated.n_weights(), np.float32)
    for name, shape, _ in gated.weight_shapes():
        if name in Pb:
            v = Pb[name].copy()
            if name.startswith("Wmix."):
                v[1:] *= 2.0  # sigmoid(0) = 1/2 on the l > 0 updates
            wg = _split_set(gated, wg, name, v)
    s = synth.cluster(18, seed=2, side=5.5)
    rb = oracle.Model(base, wb).energy_forces(s.pos, s.species, s.cell, s.pbc)
    rg = oracle.Model(gated, wg).energy_forces(s.pos, s.species, s.cell, s.pbc)
    assert abs(rb["energy"] - rg["energy"]) < 1e-12 * abs(rb["energy"])
    np.testing.assert_allclose(rg["forces"], rb["forces"], rtol=0, atol=1e-12 * np.abs(rb["forces"]).max())


def test_isolated_atom_is_the_self_connection_chain():
    spec = synth.ModelSpec(S=4, T=2, C=8, L=2, H=16, avg_nb=10.0, gate=1)
    w = synth.make_weights(spec, 23).copy()
    w[-4:] = np.array([0.3, -0.1, 0.2, 0.05], np.float32)  # E0
    P = synth.split_weights(spec, w)
    m = oracle.Model(spec, w)
    silu = lambda a: a / (1 + np.exp(-a))
    for z in range(4):
        h = P["W_emb"][z].astype(np.float64)
        for t in range(2):
            h = h + silu(h @ P[f"Wself.{t}"][z, 0].astype(np.float64))
        want = P["W_out"][z].astype(np.float64) @ h + float(P["E0"][z])
        out = m.energy_forces(np.zeros((1, 3)), np.array([z], np.int32), np.eye(3), np.zeros(3, np.uint8))
        assert abs(out["energy"] - want) < 1e-13 * max(1.0, abs(want))
        assert np.abs(out["forces"]).max() == 0.0
