"""Standard Model particle and vertex table for the process compiler.

The vertex set is the one the paper's HEGET functions cover (Sect. 4.2,
Table 2): FFV, FFS, VVV, VVVV, VVS, VVSS, SSS, SSSS.  Conventions: every vertex lists the fields
it annihilates, i.e. all particles incoming.  Couplings follow the textbook
Lagrangian with D_mu = d_mu - i g_s t^a G^a_mu - i g W^a T^a - i g' Y B_mu
(the paper's Eqs. 22-40 up to the sign convention of g_s, which drops out
of |M|^2):

  f~ f V    i gamma^mu (gL P_L + gR P_R)         photon: gL = gR = e Q
                                                 Z: gL = gZ (T3 - Q sw^2), gR = -gZ Q sw^2
                                                 W: gL = g / sqrt2, gR = 0
                                                 gluon: gL = gR = g_s, colour t^a
  g g g     g_s f^{abc} [g^{mn}(k1-k2)^r + cyclic]   (all momenta incoming)
  W+ W- V   -i g_V [g^{mn}(k1-k2)^r + cyclic] for incoming (W+, W-, V), g_A = e, g_Z = g cw
  g g g g   -i g_s^2 f^{XYe} f^{ZWe} (g_XZ g_YW - g_XW g_YZ) for the three pairings
  W+ W- h   i g mW g^{mn}        Z Z h  i gZ mZ g^{mn}
  W+ W- h h i g^2/2 g^{mn}       Z Z h h i gZ^2/2 g^{mn}
  h h h     -i 3 mH^2 / v          h h h h  -i 3 mH^2 / v^2
  t~ t h    -i mt / v
"""
import math
from dataclasses import dataclass, field


@dataclass(frozen=True)
class Particle:
    name: str
    anti: str
    spin: int          # 0, 1 (fermion) or 2 (vector): twice the spin
    colour: int        # 1, 3 (quark), -3 (antiquark) or 8
    mass: str          # parameter name or "0"
    width: str         # parameter name or "0"
    charge3: int       # 3 x electric charge
    pdg: int

    @property
    def is_fermion(self):
        return self.spin == 1

    @property
    def is_vector(self):
        return self.spin == 2

    @property
    def is_scalar(self):
        return self.spin == 0

    @property
    def massless(self):
        return self.mass == "0"


def _fermion(name, anti, colour, mass, width, charge3, pdg):
    return [Particle(name, anti, 1, colour, mass, width, charge3, pdg),
            Particle(anti, name, 1, -colour if colour == 3 else colour, mass, width, -charge3, -pdg)]


PARTICLES = {}
for p in (
    _fermion("u", "u~", 3, "0", "0", 2, 2) + _fermion("d", "d~", 3, "0", "0", -1, 1)
    + _fermion("c", "c~", 3, "0", "0", 2, 4) + _fermion("s", "s~", 3, "0", "0", -1, 3)
    + _fermion("b", "b~", 3, "0", "0", -1, 5) + _fermion("t", "t~", 3, "MT", "WT", 2, 6)
    + _fermion("e-", "e+", 1, "0", "0", -3, 11) + _fermion("ve", "ve~", 1, "0", "0", 0, 12)
    + _fermion("mu-", "mu+", 1, "0", "0", -3, 13) + _fermion("vm", "vm~", 1, "0", "0", 0, 14)
    + [Particle("g", "g", 2, 8, "0", "0", 0, 21), Particle("a", "a", 2, 1, "0", "0", 0, 22),
       Particle("z", "z", 2, 1, "MZ", "WZ", 0, 23),
       Particle("w+", "w-", 2, 1, "MW", "WW", 3, 24), Particle("w-", "w+", 2, 1, "MW", "WW", -3, -24),
       Particle("h", "h", 0, 1, "MH", "WH", 0, 25)]
):
    PARTICLES[p.name] = p

ALIASES = {"e+": "e+", "e-": "e-", "ve": "ve", "ve~": "ve~", "H": "h", "W+": "w+", "W-": "w-", "Z": "z", "A": "a"}

QUARK_T3 = {"u": 0.5, "c": 0.5, "t": 0.5, "d": -0.5, "s": -0.5, "b": -0.5, "e-": -0.5, "mu-": -0.5,
            "ve": 0.5, "vm": 0.5}
CHARGE = {"u": 2 / 3, "c": 2 / 3, "t": 2 / 3, "d": -1 / 3, "s": -1 / 3, "b": -1 / 3, "e-": -1.0, "mu-": -1.0,
          "ve": 0.0, "vm": 0.0}
WEAK_DOUBLETS = [("u", "d"), ("c", "s"), ("t", "b"), ("ve", "e-"), ("vm", "mu-")]


@dataclass(frozen=True)
class Vertex:
    """A Feynman rule: incoming fields, Lorentz kind and coupling names.

    kind: "FFV" (fields f~, f, V), "FFS" (f~, f, S), "VVV", "VVVV", "VVS", "VVSS", "SSS", "SSSS".
    couplings: names resolved by couplings() at me_create time; for FFV
    (gL, gR).  colour: "delta" (f~ f), "T" (f~ f g), "f" (ggg), "ff" (gggg).
    pair: for a colourless VVVV vertex, the slot pairing (0: (01)(23), 1: (02)(13), 2: (03)(12))
    whose metric product enters with -2 while the other two enter with +1.
    """
    fields: tuple
    kind: str
    couplings: tuple
    colour: str = "none"
    phase: int = -1   # power of i of the vertex factor; -1: the default of its kind
    pair: int = -1


def _ffv_vertices():
    out = []
    coloured = {"u", "d", "c", "s", "b", "t"}
    for f in ["u", "d", "c", "s", "b", "t", "e-", "mu-"]:
        fb = PARTICLES[f].anti
        col = "delta" if f in coloured else "none"
        out.append(Vertex((fb, f, "a"), "FFV", (f"GA_{f}", f"GA_{f}"), col))
        out.append(Vertex((fb, f, "z"), "FFV", (f"GZL_{f}", f"GZR_{f}"), col))
        if f in coloured:
            out.append(Vertex((fb, f, "g"), "FFV", ("GS", "GS"), "T"))
    for f in ["ve", "vm"]:
        out.append(Vertex((PARTICLES[f].anti, f, "z"), "FFV", (f"GZL_{f}", f"GZR_{f}"), "none"))
    for up, dn in WEAK_DOUBLETS:
        col = "delta" if up in {"u", "c", "t"} else "none"
        # u~ d W+ and d~ u W- (all incoming)
        out.append(Vertex((PARTICLES[up].anti, dn, "w+"), "FFV", ("GW", "ZERO"), col))
        out.append(Vertex((PARTICLES[dn].anti, up, "w-"), "FFV", ("GW", "ZERO"), col))
    return out


VERTICES = _ffv_vertices() + [
    Vertex(("g", "g", "g"), "VVV", ("GS",), "f"),
    Vertex(("g", "g", "g", "g"), "VVVV", ("GS2",), "ff"),
    # W W gamma and W W Z (Sect. 4.2 VVV with (V1, V2, V3) = (W-, W+, V) named by their outgoing
    # quantum numbers, i.e. incoming W+, W-, V here): -i g_V times the Lorentz structure
    Vertex(("w+", "w-", "a"), "VVV", ("GWWA",), "none", phase=3),
    Vertex(("w+", "w-", "z"), "VVV", ("GWWZ",), "none", phase=3),
    # electroweak quartic vertices (Sect. 4.2 VVVV, the W W W W and W W W3 W3 terms with each
    # vertex's two channels summed): i C [g^{ab} g^{cd} summed over the two pairings other than
    # `pair`, minus twice the metric product of `pair`]; C = -g^2 for W+ W- W+ W- (pair: the two
    # like-charged bosons) and g^2 times the W3 projections for W+ W- V V' (pair: W W and V V')
    Vertex(("w+", "w-", "w+", "w-"), "VVVV", ("GWWWW",), "none", phase=1, pair=1),
    Vertex(("w+", "w-", "a", "a"), "VVVV", ("GWWAA",), "none", phase=1, pair=0),
    Vertex(("w+", "w-", "a", "z"), "VVVV", ("GWWAZ",), "none", phase=1, pair=0),
    Vertex(("w+", "w-", "z", "z"), "VVVV", ("GWWZZ",), "none", phase=1, pair=0),
    Vertex(("w+", "w-", "h"), "VVS", ("GWWH",)),
    # top Yukawa (Sect. 4.2 FFS): L = -(mt/v) t~ t H, i (gL P_L + gR P_R) with gL = gR = -mt/v
    Vertex(("t~", "t", "h"), "FFS", ("GHTT", "GHTT"), "delta"),
    Vertex(("z", "z", "h"), "VVS", ("GZZH",)),
    Vertex(("w+", "w-", "h", "h"), "VVSS", ("GWWHH",)),
    Vertex(("z", "z", "h", "h"), "VVSS", ("GZZHH",)),
    Vertex(("h", "h", "h"), "SSS", ("GHHH",)),
    Vertex(("h", "h", "h", "h"), "SSSS", ("GHHHH",)),
]


DEFAULT_PARAMS = dict(alpha=1.0 / 128.0, sw2=0.2312, mZ=91.1876, wZ=2.4952, mW=80.4, wW=2.085,
                      alpha_s=0.118, mt=175.0, wt=1.50, mH=125.0, wH=0.0, complex_mass=0)

# couplings that carry a vector-boson mass (directly or through v = 2 mW / g): complex under the
# complex-mass option, so the generated programs take them as complex numbers (name.re, name.im)
COMPLEX_COUPLINGS = frozenset({"GWWH", "GZZH", "GHHH", "GHHHH", "GHTT"})


def couplings(par):
    """Numerical couplings, masses and widths for a parameter dict (electroweak
    scheme: e = sqrt(4 pi alpha), g = e/sw, gZ = e/(sw cw), v = 2 mW / g).

    With par["complex_mass"] (Sect. 7.11): mu_V^2 = m_V^2 - i m_V Gamma_V in the couplings, the W
    tied to the Z by mu_W^2 = cw^2 mu_Z^2 (so MW = cw mZ, WW = cw wZ), and v = 2 mu_W / g.  The
    couplings of COMPLEX_COUPLINGS appear as name.re and name.im (imaginary part 0 without the
    option)."""
    e = math.sqrt(4 * math.pi * par["alpha"])
    sw = math.sqrt(par["sw2"])
    cw = math.sqrt(1 - par["sw2"])
    g = e / sw
    gz = e / (sw * cw)
    gs = math.sqrt(4 * math.pi * par["alpha_s"])
    cms = bool(par.get("complex_mass", 0))
    mW, wW = (cw * par["mZ"], cw * par["wZ"]) if cms else (par["mW"], par["wW"])
    muW = complex(mW * mW, -mW * wW) ** 0.5 if cms else complex(mW)
    muZ = complex(par["mZ"] ** 2, -par["mZ"] * par["wZ"]) ** 0.5 if cms else complex(par["mZ"])
    v = 2 * muW / g
    c = {"ZERO": 0.0, "GS": gs, "GS2": gs * gs, "GW": g / math.sqrt(2),
         "GWWHH": g * g / 2, "GZZHH": gz * gz / 2,
         "GWWA": e, "GWWZ": g * cw,
         "GWWWW": -g * g, "GWWAA": g * g * sw * sw, "GWWAZ": g * g * sw * cw, "GWWZZ": g * g * cw * cw,
         "MT": par["mt"], "WT": par["wt"], "MZ": par["mZ"], "WZ": par["wZ"], "MW": mW, "WW": wW,
         "MH": par["mH"], "WH": par["wH"], "0": 0.0}
    cplx = {"GWWH": g * muW, "GZZH": gz * muZ, "GHHH": -3 * par["mH"] ** 2 / v, "GHTT": -par["mt"] / v,
            "GHHHH": -3 * par["mH"] ** 2 / v ** 2}
    for n, z in cplx.items():
        c[n + ".re"], c[n + ".im"] = z.real, z.imag
    for f, q in CHARGE.items():
        c[f"GA_{f}"] = e * q
        c[f"GZL_{f}"] = gz * (QUARK_T3[f] - q * par["sw2"])
        c[f"GZR_{f}"] = gz * (-q * par["sw2"])
    return c
