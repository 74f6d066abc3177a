"""Plant plausible mistakes in copies of the oracle (on the CPU) and check
that the pins catch every one of them: a dropped term, a wrong sign, an
off-by-one in the half-open interval of Algorithm 2, swapped interpolation
weights, a wrong power of the Doppler factor, a wrong spectral prefactor,
a transposed operand, a wrong grid bound."""
import os

import pytest

import oracle
import oracle_pins
from oracle import oracle as _orc

MUTATIONS = {
    "cross_sign": ("out[0] = a[1] * b[2] - a[2] * b[1];", "out[0] = a[1] * b[2] + a[2] * b[1];"),
    "cross_transposed": ("cross3(n, inner, outer);", "cross3(inner, n, outer);"),
    "doppler_power": ("double D3 = D * D * D;", "double D3 = D * D;"),
    "weights_swapped": ("out[c * n_bins + j] += Eb[3 * k + c] * wa + E[c] * wb;",
                        "out[c * n_bins + j] += Eb[3 * k + c] * wb + E[c] * wa;"),
    "buffer_unused": ("out[c * n_bins + j] += Eb[3 * k + c] * wa + E[c] * wb;",
                      "out[c * n_bins + j] += E[c] * wa + E[c] * wb;"),
    "interval_closed_left": ("int64_t j_lo = (int64_t)floor(ub) + 1;",
                             "int64_t j_lo = (int64_t)floor(ub);"),
    "interval_open_right": ("int64_t j_hi = (int64_t)floor(ua);",
                            "int64_t j_hi = (int64_t)floor(ua) - 1;"),
    "time_map_sign": ("return t - nr * inv_c0;", "return t + nr * inv_c0;"),
    "time_map_dropped_z": ("nr = nr + n[2] * r[2];", "nr = nr + 0.0 * r[2];"),
    "grid_point_offset": ("double tu = t_min + (double)j * dt_u;",
                          "double tu = t_min + ((double)j + 0.5) * dt_u;"),
    "component_index": ("out[c * n_bins + j] +=", "out[j] +="),
    "fft_sign": ("double wr = cos(ang), wi = sin(ang);", "double wr = cos(ang), wi = -sin(ang);"),
    "spectrum_prefactor": ("const double scale = K * dt_u * dt_u;", "const double scale = K * dt_u;"),
    "spectrum_pi_power": (
        "const double K = q * q / (16.0 * OR_PI * OR_PI * OR_PI * OR_EPS0 * OR_C0);\n"
        "    const double scale",
        "const double K = q * q / (16.0 * OR_PI * OR_PI * OR_EPS0 * OR_C0);\n"
        "    const double scale"),
    "velocity_gamma": ("double g = OR_C0 * (1.0 - b2) / (D3 * dist);",
                       "double g = OR_C0 / (D3 * dist);"),
    "exact_distance": ("scale = R / dist;", "scale = 1.0;"),
    "grid_min_at_end": ("if (a0 < lo) lo = a0;", "if (a1 < lo) lo = a1;"),
    "fdm_doppler_power": ("double a = A[c] / (D * D);", "double a = A[c] / D;"),
    "clip_silent": ("if (a < 0) { a = 0; st |= ST_CLIP; }", "if (a < 0) { a = 0; }"),
    "grad_t_a_sign": ("gta += Rc * (Eb[c] - E[c]) * (tu - tb) / (den * den);",
                      "gta -= Rc * (Eb[c] - E[c]) * (tu - tb) / (den * den);"),
    "grad_weights_swapped": ("gEb[c] += Rc * (ta - tu) / den;", "gEb[c] += Rc * (tu - tb) / den;"),
    "grad_doppler_term": ("s += 3.0 * n[d] * dot3(gE, E) / D;", "s += 2.0 * n[d] * dot3(gE, E) / D;"),
    "grad_time_map_sign": ("o_r[d] += -gta * n[d] / OR_C0;", "o_r[d] += gta * n[d] / OR_C0;"),
    "grad_conjugate": ("acc += g[m * nl + l] * 2.0 * (Xre[l] * cos(ang) + Xim[l] * sin(ang));",
                       "acc += g[m * nl + l] * 2.0 * (Xre[l] * cos(ang) - Xim[l] * sin(ang));"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = _orc.source_text()
    assert src.count(old) >= 1, f"mutation anchor missing: {old!r}"
    path = os.path.join(str(tmp_path), f"liboracle_{name}.so")
    _orc.build_variant(src.replace(old, new, 1), path)
    caught = []
    with _orc.use_library(path):
        for pin in oracle_pins.ALL_PINS:
            try:
                pin()
            except Exception:  # noqa: BLE001 - any failure counts as caught
                caught.append(pin.__name__)
    assert caught, f"no pin caught mutation {name}"
