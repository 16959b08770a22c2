"""Standard Model parameter card and Feynman-rule couplings for the oracle.

Oracle module (test infrastructure only).  Default inputs are the workload
inputs: alpha = 1/128, sin^2(theta_W) = 0.2312, mZ = 91.1876, GammaZ = 2.4952,
mW = 80.4, GammaW = 2.085, alpha_s = 0.118, mt = 175, Gammat = 1.50, mH = 125.

Electroweak scheme (the paper leaves the scheme to the generator; Sect. 7.11
discusses its effect on HHH): e = sqrt(4 pi alpha), g = e / s_W,
g_Z = e / (s_W c_W), v = 2 mW / g.

Complex-mass option (Sect. 7.11; the card's cms flag, made by with_cms()): every
vector-boson mass in propagators and couplings becomes mu_V with mu_V^2 = m_V^2 - i m_V
Gamma_V, and the W is tied to the Z by the tree-level relation mu_W^2 = c_W^2 mu_Z^2
(m_W = c_W m_Z, Gamma_W = c_W Gamma_Z).  The couplings that carry a boson mass become
complex: W W H = g mu_W, Z Z H = g_Z mu_Z, and v = 2 mu_W / g in H H H, H H H H and the
top Yukawa.  Propagator denominators q^2 - m^2 + i m Gamma and the q q / mu^2 numerator
terms are the same in both schemes.  Vertex factors are those of the
textbook Lagrangian with D_mu = d_mu - i g_s t^a A^a_mu - i g W^a T^a - i g' Y B:
  f f gamma : i e Q gamma^mu
  f f Z     : i g_Z gamma^mu (T3 P_L - Q s_W^2)
  u d W     : i g/sqrt(2) gamma^mu P_L
  q q g     : i g_s gamma^mu t^a
  W W H     : i g mW g^{mu nu}          W W H H : i g^2/2 g^{mu nu}
  H H H     : -i 3 mH^2 / v
"""
import math
from dataclasses import dataclass, replace


@dataclass(frozen=True)
class SMParams:
    alpha: float = 1.0 / 128.0
    sw2: float = 0.2312
    mZ: float = 91.1876
    wZ: float = 2.4952
    mW: float = 80.4
    wW: float = 2.085
    alpha_s: float = 0.118
    mt: float = 175.0
    wt: float = 1.50
    mH: float = 125.0
    wH: float = 0.0
    cms: bool = False

    @property
    def e(self):
        return math.sqrt(4.0 * math.pi * self.alpha)

    @property
    def sw(self):
        return math.sqrt(self.sw2)

    @property
    def cw(self):
        return math.sqrt(1.0 - self.sw2)

    @property
    def g(self):
        return self.e / self.sw

    @property
    def gz(self):
        return self.e / (self.sw * self.cw)

    @property
    def gs(self):
        return math.sqrt(4.0 * math.pi * self.alpha_s)

    @property
    def muW(self):
        """W mass in couplings: m_W, or sqrt(m_W^2 - i m_W Gamma_W) (principal root) with cms."""
        if not self.cms:
            return self.mW
        return complex(self.mW * self.mW, -self.mW * self.wW) ** 0.5

    @property
    def muZ(self):
        if not self.cms:
            return self.mZ
        return complex(self.mZ * self.mZ, -self.mZ * self.wZ) ** 0.5

    @property
    def vev(self):
        return 2.0 * self.muW / self.g

    @property
    def gwwh(self):
        return self.g * self.muW

    @property
    def gzzh(self):
        return self.gz * self.muZ

    def with_(self, **kw):
        return replace(self, **kw)

    def with_cms(self):
        """The complex-mass card: the flag set and the W mass and width tied to the Z's."""
        return replace(self, cms=True, mW=self.cw * self.mZ, wW=self.cw * self.wZ)


# electric charge and weak isospin of the fermions used here
CHARGE = {"u": 2 / 3, "c": 2 / 3, "t": 2 / 3, "d": -1 / 3, "s": -1 / 3, "b": -1 / 3, "e": -1.0, "ve": 0.0}
T3 = {"u": 0.5, "c": 0.5, "t": 0.5, "d": -0.5, "s": -0.5, "b": -0.5, "e": -0.5, "ve": 0.5}

GEV2_TO_PB = 0.3893793721e9
