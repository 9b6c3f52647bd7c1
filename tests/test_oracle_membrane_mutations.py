"""Plausible mistakes planted in the membrane oracle must fail its pins.

Each mutation replaces one step of oracle/membrane.py (monkeypatched, CPU
only) and runs the pins of tests/test_oracle_membrane.py that cover it; at
least one must fail.
"""

import numpy as np
import pytest

import test_oracle_membrane as pins
from oracle import membrane as mb

_orig_jac = mb.transition_jacobian
_orig_tension = mb.skalak_tension
_orig_div = mb.divergence_from


def transposed_jacobian(i, j, u, v):
    return np.swapaxes(_orig_jac(i, j, u, v), -1, -2)


def _parts(geo, ref):
    N = geo["xu"].shape[0]
    A = np.stack([ref["xu"], ref["xv"], ref["n"]], axis=-1)
    B = np.stack([geo["xu"], geo["xv"], np.zeros((N, 3))], axis=-1)
    Fs = B @ np.linalg.inv(A)
    V2 = Fs @ np.swapaxes(Fs, -1, -2)
    ev = np.sort(np.linalg.eigvalsh(V2), axis=-1)[:, 1:]
    I1 = ev[:, 0] + ev[:, 1] - 2.0
    I2 = ev[:, 0] * ev[:, 1] - 1.0
    Js = np.sqrt(ev[:, 0] * ev[:, 1])
    n = geo["n"]
    P = np.eye(3)[None] - n[:, :, None] * n[:, None, :]
    return V2, I1, I2, Js, P


def tension_js_inverted(geo, ref, Es, ED):
    """Es / (2 J_s) written as Es J_s / 2."""
    V2, I1, I2, Js, P = _parts(geo, ref)
    return ((Es * Js / 2 * (I1 + 1))[:, None, None] * V2
            + (0.5 * Js * (ED * I2 - Es))[:, None, None] * P)


def tension_drop_plus_one(geo, ref, Es, ED):
    """(I1 + 1) V^2 written as I1 V^2."""
    V2, I1, I2, Js, P = _parts(geo, ref)
    return ((Es / (2 * Js) * I1)[:, None, None] * V2
            + (0.5 * Js * (ED * I2 - Es))[:, None, None] * P)


def tension_ref_current_swapped(geo, ref, Es, ED):
    return _orig_tension(ref, geo, Es, ED)


def divergence_E_G_swapped(geo, gu, gv):
    g2 = dict(geo)
    g2["E"], g2["G"] = geo["G"], geo["E"]
    return _orig_div(g2, gu, gv)


def blend_own_psi(m, du, dv):
    """Blending that weights every patch by the node's own-patch psi_i."""
    from capsule_inputs.geometry import chart, pou_all
    n, h, F = m - 1, np.pi / m, du.shape[-1]
    j_, k_ = np.meshgrid(np.arange(1, m), np.arange(1, m), indexing="ij")
    u, v = (j_ * h).ravel(), (k_ * h).ravel()
    out_u = np.zeros((6, n * n, F))
    out_v = np.zeros_like(out_u)
    for i in range(1, 7):
        psi = pou_all(chart(i, u, v))
        out_u[i - 1] = psi[:, i - 1, None] * du[i - 1].reshape(-1, F)
        out_v[i - 1] = psi[:, i - 1, None] * dv[i - 1].reshape(-1, F)
        for p in range(1, 7):
            sel = (psi[:, p - 1] > 0.0) & (p != i)
            if not np.any(sel):
                continue
            up, vp = mb.transition(i, p, u[sel], v[sel])
            Iu = mb.interpolate(m, du[p - 1], up, vp)
            Iv = mb.interpolate(m, dv[p - 1], up, vp)
            J = mb.transition_jacobian(i, p, u[sel], v[sel])
            w = psi[sel, i - 1][:, None]          # mistake: psi_i instead of psi_p
            out_u[i - 1, sel] += w * (Iu * J[:, 0, 0, None] + Iv * J[:, 0, 1, None])
            out_v[i - 1, sel] += w * (Iu * J[:, 1, 0, None] + Iv * J[:, 1, 1, None])
    return out_u.reshape(6 * n * n, F), out_v.reshape(6 * n * n, F)


MUTATIONS = {
    "transposed_jacobian": ("transition_jacobian", transposed_jacobian),
    "blend_own_psi": ("blend", blend_own_psi),
    "tension_js_inverted": ("skalak_tension", tension_js_inverted),
    "tension_drop_plus_one": ("skalak_tension", tension_drop_plus_one),
    "tension_ref_current_swapped": ("skalak_tension", tension_ref_current_swapped),
    "divergence_E_G_swapped": ("divergence_from", divergence_E_G_swapped),
    "stencil_outer_terms_dropped": ("FD7", np.array([0.0, 9.0, -45.0, 0.0, 45.0, -9.0, 0.0]) / 60.0),
}

PINS = [
    lambda: pins.test_sphere_derivatives_at_or_below_printed_errors(16),
    pins.test_ellipsoid_derivatives_printed_table_and_fourth_order,
    pins.test_uniform_dilation_of_a_sphere_closed_form,
    pins.test_virtual_work_matches_skalak_energy_variation,
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_fails_a_pin(name, monkeypatch):
    attr, repl = MUTATIONS[name]
    monkeypatch.setattr(mb, attr, repl)
    failed = 0
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                pin()
        except (AssertionError, np.linalg.LinAlgError):  # a pin that cannot run fails
            failed += 1
    assert failed >= 1, f"mutation {name} passed every pin"


def test_unmutated_oracle_passes_the_same_pins():
    for pin in PINS:
        pin()
