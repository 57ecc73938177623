"""Gradient-based scaling of the AL problem (TEST INFRASTRUCTURE ONLY).

Sec. IV-A "Scaling": the objective is scaled by sigma_f and constraint i by
sigma_c[i] so that their magnitudes match; the paper names the rule (scale by
the size of the gradient, as interior-point codes do) without writing it out.
The reading taken here is the usual gradient-based rule of those codes, over
the controls u and with the reduced derivatives on g = 0:

    scale(n)   = 1 if n <= g_max, else max(s_min, g_max / n)
    sigma_c[i] = p_i scale(p_i ||dc_i/du||_inf)

where p_i is the caller's own scale of constraint i (1 without one: the rule
then applies to the constraint as the caller writes it, p_i c_i, as
interior-point codes apply it to the model as given), and sigma_f =
scale(||df/du||_inf) with the reduced gradient of the generation cost
(Prop. 1 with sigma_f = 1 and no multiplier or penalty term).  J = dc/du is
the oracle's explicit reduced Jacobian (one Jacobian-vector product per
control, `explicit_jacobian`).
"""
import numpy as np


def scale_of(norm, g_max=100.0, s_min=1e-8):
    """The scale of a function whose largest derivative magnitude is `norm` (array or scalar)."""
    norm = np.asarray(norm, dtype=np.float64)
    out = np.ones_like(norm)
    big = norm > g_max
    out[big] = np.maximum(s_min, g_max / norm[big])
    return out


def gradient_scaling(J, grad_f, g_max=100.0, s_min=1e-8, prior=None):
    """(sigma_c [m], sigma_f) from the reduced Jacobian J (m x n_u) and the reduced cost gradient.
    With the caller's own constraint scales `prior` the rule applies to the constraints as written,
    prior_i c_i: sigma_c[i] = prior_i scale_of(prior_i ||dc_i/du||_inf)."""
    J = np.asarray(J, dtype=np.float64)
    rows = np.abs(J).max(axis=1) if J.shape[1] else np.zeros(J.shape[0])
    p = np.ones(J.shape[0]) if prior is None else np.asarray(prior, dtype=np.float64)
    gf = np.asarray(grad_f, dtype=np.float64)
    sigma_f = float(scale_of(np.abs(gf).max() if gf.size else 0.0, g_max, s_min))
    return p * scale_of(p * rows, g_max, s_min), sigma_f


def explicit_jacobian(on, x, u, pd=None, qd=None, cols=None):
    """J = dc/du on g = 0, one oracle product J e_j per requested control (all by default)."""
    cols = range(on.nu) if cols is None else cols
    J = np.zeros((on.m, len(cols)))
    for k, j in enumerate(cols):
        e = np.zeros(on.nu)
        e[j] = 1.0
        J[:, k], _ = on.jac_prod(x, u, v=e, pd=pd, qd=qd)
    return J


def cost_gradient(on, x, u, pd=None, qd=None):
    """Reduced gradient of the generation cost alone (Prop. 1 with sigma_f = 1, rho = 0, y = 0)."""
    z = np.zeros(on.m)
    al = dict(sigma_f=1.0, rho=0.0, sigma_c=z, y=z, s=z)
    return on.reduced_gradient(x, u, al, pd=pd, qd=qd)["grad_u"]
