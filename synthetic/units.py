"""Lattice-unit parameter sets for the paper's two flows.

Kolmogorov flow (Sec. 6, "Lattice units"): length scale C_l = 2*pi/N, velocity
scale C_u = U / (0.1 c_s*) with U = 4 and c_s* = 1/sqrt(3), density scale 1.
The time scale is C_t = C_l / C_u, so one time unit (TU) is C_u / C_l steps.
The non-dimensional viscosity 1/Re becomes nu* = (1/Re) C_t / C_l**2, the
forcing amplitude 1 becomes C_t / C_u, and the linear drag rate 0.1 becomes
0.1 C_t per step.

Channel flow (Sec. 7.1, setup): C_l = 2H / (N_y - 2) (one solid layer per wall),
centre-line velocity U_c+ maps to 0.1 lattice units, so u_tau* = 0.1 / U_c+.
Re_tau = u_tau H / nu fixes nu*, and the driving body force that balances the
wall shear is F = u_tau**2 / H.  One TU is H / u_tau steps.

The paper states U_c+ ~ 18.3 but also gives 4289 LF steps per TU at N_y = 49;
U_c+ = 18.25 reproduces that count (and 21 445 HF steps within 0.01 %), so it
is the default here.
"""

import math

CS = 1.0 / math.sqrt(3.0)


def kolmogorov_lattice(n, re=1.0e4, u_char=4.0, force_amp=1.0, drag=0.1, k_forcing=4):
    c_l = 2.0 * math.pi / n
    c_u = u_char / (0.1 * CS)
    c_t = c_l / c_u
    nu = (1.0 / re) * c_t / c_l ** 2
    return dict(
        n=n,
        c_l=c_l,
        c_u=c_u,
        steps_per_tu=1.0 / c_t,
        nu=nu,
        tau=3.0 * nu + 0.5,
        kolmo_amp=force_amp * c_t / c_u,
        kolmo_drag=drag * c_t,
        kolmo_k=k_forcing,
    )


def channel_lattice(ny, re_tau=180.0, u_c=0.1, u_c_plus=18.25):
    h = 0.5 * (ny - 2)
    u_tau = u_c / u_c_plus
    nu = u_tau * h / re_tau
    return dict(
        ny=ny,
        h=h,
        u_tau=u_tau,
        nu=nu,
        tau=3.0 * nu + 0.5,
        body_force=u_tau ** 2 / h,
        steps_per_tu=h / u_tau,
        u_c=u_c,
    )
