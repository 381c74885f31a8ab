"""Parameter sets shared by the tests (plain numbers, no method arithmetic).

EOS constants a, b, R are the paper's (text after Eq. 4).  The temperature of
each case is set by the target liquid/gas density ratio; the tests obtain it
from the oracle (CPU tests) or from the library (GPU tests).
"""
A, B, RGAS = 0.037, 0.2, 1.0


def base(T, **kw):
    p = dict(a=A, b=B, R=RGAS, T=T, lambda1=0.6, lambda2=0.5, lambda3=0.5,
             kappa1=0.01, kappa2=1.0, kappa3=1.0, chi=5.0, nu=1.0 / 6.0,
             Gamma=1.0, tau_g=1.0, force_form=1)
    p.update(kw)
    return p


def asymmetric(T, **kw):
    """Unequal liquid parameters so that every cross term is exercised."""
    p = base(T, lambda2=0.4, lambda3=0.7, kappa1=0.02, kappa2=0.8, kappa3=1.3,
             nu=0.1, Gamma=0.7, tau_g=0.9)
    p.update(kw)
    return p
