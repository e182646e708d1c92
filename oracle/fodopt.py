"""FOD relaxation for the oracle (TEST INFRASTRUCTURE ONLY; see the package
header): minimise E_SIC over the FOD positions with the FOD forces (Sec. II
obtains the FODs by minimising the SIC energy with the forces of Eq. 9;
Sec. III converges every FOD to a force below 1e-3 Eh/bohr).

The paper names no minimiser; like the library this uses FIRE (Bitzek,
Koskinen, Gaehler, Moseler, Gumbsch, Phys. Rev. Lett. 97, 170201 (2006)),
unit masses, semi-implicit Euler, with the same parameters, written here in
plain NumPy for a single system:

  F = -grad E; stop when max |F| < fmax; P = F . v
  P > 0:  v = (1 - alpha) v + alpha |v| F/|F|; count this; once the count
          exceeds n_min: dt = min(f_inc dt, dt_max), alpha = f_alpha alpha
  P <= 0: v = 0, dt = f_dec dt, alpha = alpha_start, count = 0
  v = v + dt F;  x = x + dt v
"""
import numpy as np

from .flosic import sic_backward, sic_forward

FIRE_DEFAULTS = dict(dt0=0.2, dt_max=1.0, n_min=5, f_inc=1.1, f_dec=0.5, alpha0=0.1, f_alpha=0.99)


def fire(fun, x0, fmax=1e-3, max_steps=500, **params):
    """fun(x) -> (E, grad).  Returns (x, E, max|F|, steps, history of E)."""
    p = dict(FIRE_DEFAULTS)
    p.update(params)
    x = np.array(x0, dtype=np.float64)
    v = np.zeros_like(x)
    dt, alpha, count = p["dt0"], p["alpha0"], 0
    hist = []
    steps = 0
    while True:
        E, g = fun(x)
        F = -np.asarray(g, dtype=np.float64)
        hist.append(E)
        fm = float(np.max(np.abs(F)))
        if fm < fmax or steps == max_steps:
            return x, E, fm, steps, hist
        power = float(np.dot(F, v))
        if power > 0.0:
            vnorm = np.sqrt(np.dot(v, v))
            fnorm = np.sqrt(np.dot(F, F))
            v = (1.0 - alpha) * v + alpha * vnorm * F / max(fnorm, 1e-300)
            count += 1
            if count > p["n_min"]:
                dt = min(dt * p["f_inc"], p["dt_max"])
                alpha *= p["f_alpha"]
        else:
            v = np.zeros_like(x)
            dt *= p["f_dec"]
            alpha = p["alpha0"]
            count = 0
        v = v + dt * F
        x = x + dt * v
        steps += 1


def relax_fods(psi_blocks, fod_blocks, grid, fmax=1e-3, max_steps=500, scale=1.0, tol=1e-12, **params):
    """One system: FIRE over all its FODs (spins concatenated, [sum N, 3])."""
    sizes = [len(f) for f in fod_blocks]

    def fun(x):
        fb = []
        o = 0
        for n in sizes:
            fb.append(x[3 * o:3 * (o + n)].reshape(n, 3))
            o += n
        fwd = sic_forward(psi_blocks, fb, grid, scale=scale, tol=tol)
        _, dfod = sic_backward(fwd, grid)
        return fwd["E_sic"], np.concatenate([d.ravel() for d in dfod])

    x0 = np.concatenate([np.asarray(f, dtype=np.float64).ravel() for f in fod_blocks])
    return fire(fun, x0, fmax, max_steps, **params)
