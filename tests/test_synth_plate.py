"""The flat-plate input generator against textbook values (inputs only; no
method arithmetic is involved).

* Blasius: f''(0) = 0.332057 (White, Viscous Fluid Flow, Table 4-1), f' -> 1.
* Crocco-Busemann temperature: T = T_w at the wall and -> 1 in the free
  stream; T_aw = 1 + sqrt(Pr) (gamma - 1) M^2 / 2.
* Grading: first cell 1e-4 of the height, cells fill the height exactly,
  constant growth ratio.
* Tags: inflow 1, outflow 2, wall 3, top 1, periodic span.
"""
import numpy as np

import synth


def test_blasius_wall_shear():
    fp, s = synth.blasius()
    assert abs(s - 0.332057) < 2e-6
    assert abs(fp(12.0) - 1.0) < 1e-9 and fp(0.0) == 0.0


def test_grading():
    y = synth.graded_coordinates(48, 0.1, 1e-5)
    d = np.diff(y)
    assert abs(y[-1] - 0.1) < 1e-15 and abs(d[0] - 1e-5) < 1e-12
    r = d[1:] / d[:-1]
    assert np.ptp(r) < 1e-9 and 1.15 < r[0] < 1.2


def test_plate_state_and_tags():
    P = synth.config5(4, 6, 3, 2)
    g, M, pr = P.gamma, P.mach, P.pr
    t_aw = 1.0 + np.sqrt(pr) * (g - 1) * M ** 2 / 2
    assert abs(P.twall - 0.5 * t_aw) < 1e-14
    x = synth.node_xyz(P.mesh, P.p)
    rho = P.U[:, 0, :]
    wall = np.abs(x[..., 1]) < 1e-14
    assert wall.any()
    # at the wall: T = T_w, so rho = 1 / T_w (p = p_inf, T~ = gamma M^2 p / rho)
    assert np.allclose(rho[wall], 1.0 / P.twall, rtol=1e-10)
    top = np.abs(x[..., 1] - 0.1) < 1e-14
    assert np.allclose(rho[top], 1.0, rtol=1e-8)
    tags = P.mesh.bnd_tag
    assert set(np.unique(tags)) == {0, 1, 2, 3}
    assert (tags[:, 0][tags[:, 0] != 0] == 1).all() and (tags[:, 1][tags[:, 1] != 0] == 2).all()
    assert (tags[:, 2][tags[:, 2] != 0] == 3).all() and (tags[:, 3][tags[:, 3] != 0] == 1).all()
    assert (tags[:, 4:] == 0).all()
