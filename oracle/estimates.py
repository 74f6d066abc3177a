"""Closed-form estimates of the paper that size the observer grid and choose
the parallel scheme (arXiv 2206.03015, Sec. 4 and Sec. 5.2).

TEST INFRASTRUCTURE ONLY (oracle side).  Each function restates one equation
in plain arithmetic; the pins in ``tests/test_oracle_pins.py`` check them
against the numbers the paper prints (Tables 1 and 2, the break-even exponent).
"""
from __future__ import annotations

import math


def t_rad(T_laser: float, gamma: float) -> float:
    """Eq. (Tu_second): single-particle pulse length T_laser / (2 gamma^2)."""
    return T_laser / (2.0 * gamma * gamma)


def t_bunch_rad(l_x: float, l_y: float, l_z: float, gamma: float, c0: float) -> float:
    """Eq. (Tu_first): arrival-time spread bound l_x/(gamma c0) + l_y/(gamma c0) + l_z/c0."""
    return l_x / (gamma * c0) + l_y / (gamma * c0) + l_z / c0


def t_u_estimate(l_x, l_y, l_z, T_laser, gamma, c0):
    """Eq. (Tu_estimation): T_u ~ T_bunch_rad + T_rad."""
    return t_bunch_rad(l_x, l_y, l_z, gamma, c0) + t_rad(T_laser, gamma)


def n_tu_estimate(l_x, l_y, l_z, T_laser, gamma, lam0, c0):
    """Nyquist grid size from Eqs. (NTu_estimation_1..3) combined with (Tu_estimation):
    N_Tu = 2 omega_max / d_omega, omega_max = 4 gamma^2 omega_0, d_omega = 2 pi / T_u,
    i.e. N_Tu ~ 8 gamma^2 (l_x/(gamma lam0) + l_y/(gamma lam0) + l_z/lam0
                           + c0 T_laser/(2 gamma^2 lam0))."""
    omega0 = 2.0 * math.pi * c0 / lam0
    omega_max = 4.0 * gamma * gamma * omega0
    T_u = t_u_estimate(l_x, l_y, l_z, T_laser, gamma, c0)
    d_omega = 2.0 * math.pi / T_u
    return 2.0 * omega_max / d_omega


def n_tu_estimate_closed(l_x, l_y, l_z, T_laser, gamma, lam0, c0):
    """The same estimate in the closed form printed after Eq. (NTu_estimation_3)."""
    g2 = gamma * gamma
    return 8.0 * g2 * (l_x / (gamma * lam0) + l_y / (gamma * lam0) + l_z / lam0
                       + c0 * T_laser / (2.0 * g2 * lam0))


def phi_memory_ratio(P, N_p, N_obs, N_Tu):
    """Eq. (parallel_scheme_function), first form: M_beam / M_detector."""
    m_beam = 12.0 * N_p / P + N_obs * (4.0 * N_p / P + 3.0 * N_Tu)
    m_det = 12.0 * N_p + N_obs / P * (4.0 * N_p + 3.0 * N_Tu)
    return m_beam / m_det


def phi_memory_ratio_expanded(P, N_p, N_obs, N_Tu):
    """Eq. (parallel_scheme_function), second form."""
    num = 3.0 * (1.0 - 1.0 / P) * (N_obs * N_Tu - 4.0 * N_p)
    den = 12.0 * N_p + N_obs / P * (4.0 * N_p + 3.0 * N_Tu)
    return 1.0 + num / den


def fdm_breakeven_exponent(C_omega, C2_t, N_s, N_p):
    """Exponent of the break-even condition after Eq. (performance_model_ratio):
    N_omega > 0.5 exp(0.5 (C_omega / C2_t) N_s N_p); 'log' is the natural log."""
    return 0.5 * (C_omega / C2_t) * N_s * N_p


def wallclock_tdm(C1_t, C2_t, N_s, N_p, N_obs, N_Tu):
    """Wall-clock model W1_t + W2_t of Sec. 5.2 (natural log)."""
    return C1_t * N_s * N_p * N_obs, C2_t * N_obs * N_Tu * math.log(N_Tu)
