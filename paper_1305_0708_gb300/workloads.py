"""The benchmark workloads: process, phase-space generator, cuts, size, seed.

Each entry mirrors one workload configuration: the process string compiled
into the library, the me_kin fields of its generator and cuts, the number of
accepted points and the seed.  The oracle tests read the same numbers and
pass them to the oracle's own generator.
"""
import math

WORKLOADS = {
    "uux_epem": dict(
        process="u u~ > e+ e-", kind="two_body", sqrt_s=500.0, n=65536, seed=0, cuts=None, s_ident=1.0,
        describe="u u~ > e+ e- via photon and Z, sqrt(s)=500 GeV, cos(theta) and phi uniform, 65,536 points, seed 0"),
    "udx_epvegg": dict(
        process="u d~ > e+ ve g g", kind="rambo", sqrt_s=1000.0, n=1 << 20, seed=1,
        cuts=dict(legs=(2, 4, 5), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=0.5,
        describe="u d~ > e+ ve g g (W+ -> e+ ve plus two gluons), RAMBO at sqrt(s)=1 TeV, pT>20, |eta|<2.5, "
                 "DeltaR>0.4 on g, g, e+, 2^20 accepted points, seed 1"),
    "gg_ttx_dilep": dict(
        process="g g > (t > b (w+ > e+ ve)) (t~ > b~ (w- > e- ve~))", kind="ttbar", sqrt_s_range=(400.0, 2000.0),
        n=1 << 20, seed=2, cuts=None, s_ident=1.0,
        describe="g g > t t~ > b e+ ve b~ e- ve~, sqrt(s) uniform in [400, 2000] GeV, Breit-Wigner t and W, "
                 "isotropic decays, 2^20 points, seed 2"),
    "gg_gggg": dict(
        process="g g > g g g g", kind="rambo", sqrt_s=1500.0, n=1 << 18, seed=3,
        cuts=dict(legs=(2, 3, 4, 5), pt_min=30.0, eta_max=2.5, dr_min=0.4), s_ident=1.0 / 24.0,
        describe="g g > g g g g (six gluons, 120 colour orderings), RAMBO at sqrt(s)=1.5 TeV, pT>30, |eta|<2.5, "
                 "DeltaR>0.4 on the four final gluons, 2^18 accepted points, seed 3"),
    "us_dchh": dict(
        process="u s > d c h h", kind="rambo", sqrt_s=1000.0, masses=(0, 0, 0, 0, 125.0, 125.0), n=1 << 18, seed=4,
        cuts=None, s_ident=0.5,
        describe="u s > d c h h (W+ W- fusion), massive RAMBO at sqrt(s)=1 TeV, 2^18 points, seed 4"),
}

# The same processes with another generator (not part of the benchmark workload list)
VARIANTS = {
    "udx_epvegg_bw": dict(
        process="u d~ > e+ ve g g", kind="rambo_bw", sqrt_s=1000.0, res_mass=80.4, res_width=2.085, n=1 << 20,
        seed=1, cuts=dict(legs=(2, 4, 5), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=0.5,
        describe="u d~ > e+ ve g g with the W+ -> e+ ve pair generated Breit-Wigner mapped (App. A.2) and "
                 "RAMBO for (W*, g, g) at sqrt(s)=1 TeV, same cuts, 2^20 points, seed 1"),
    "uux_wpwm": dict(
        process="u u~ > w+ w-", kind="rambo", sqrt_s=500.0, masses=(0, 0, 80.4, 80.4), n=1 << 20, seed=5,
        cuts=None, s_ident=1.0,
        describe="u u~ > W+ W- (t-channel d, s-channel photon and Z through the WWV vertex), massive RAMBO "
                 "at sqrt(s)=500 GeV, 2^20 points, seed 5"),
    "udx_wpz": dict(
        process="u d~ > w+ z", kind="rambo", sqrt_s=500.0, masses=(0, 0, 80.4, 91.1876), n=1 << 20, seed=6,
        cuts=None, s_ident=1.0,
        describe="u d~ > W+ Z (u and d exchange, s-channel W through the WWZ vertex), massive RAMBO at "
                 "sqrt(s)=500 GeV, 2^20 points, seed 6"),
    "udx_wpa": dict(
        process="u d~ > w+ a", kind="rambo", sqrt_s=500.0, masses=(0, 0, 80.4, 0), n=1 << 20, seed=27,
        cuts=dict(legs=(3,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u d~ > W+ gamma (photon from either quark and from the s-channel W through the WWA vertex), "
                 "massive RAMBO at sqrt(s)=500 GeV, photon pT>20, |eta|<2.5, 2^20 accepted points, seed 27"),
    "uux_za": dict(
        process="u u~ > z a", kind="rambo", sqrt_s=500.0, masses=(0, 0, 91.1876, 0), n=1 << 20, seed=28,
        cuts=dict(legs=(3,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u u~ > Z gamma, massive RAMBO at sqrt(s)=500 GeV, photon pT>20, |eta|<2.5, 2^20 accepted "
                 "points, seed 28"),
    "uux_aa": dict(
        process="u u~ > a a", kind="rambo", sqrt_s=500.0, n=1 << 20, seed=29,
        cuts=dict(legs=(2, 3), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=0.5,
        describe="u u~ > gamma gamma (identical photons), RAMBO at sqrt(s)=500 GeV, pT>20, |eta|<2.5, "
                 "DeltaR>0.4 on the photons, 2^20 accepted points, seed 29"),
    "uux_zz": dict(
        process="u u~ > z z", kind="rambo", sqrt_s=500.0, masses=(0, 0, 91.1876, 91.1876), n=1 << 20, seed=7,
        cuts=None, s_ident=0.5,
        describe="u u~ > Z Z (t- and u-channel u exchange, identical Z bosons), massive RAMBO at "
                 "sqrt(s)=500 GeV, 2^20 points, seed 7"),
    "uux_zh": dict(
        process="u u~ > z h", kind="rambo", sqrt_s=500.0, masses=(0, 0, 91.1876, 125.0), n=1 << 20, seed=8,
        cuts=None, s_ident=1.0,
        describe="u u~ > Z H (s-channel Z, ZZH vertex), massive RAMBO at sqrt(s)=500 GeV, 2^20 points, seed 8"),
    "udx_wph": dict(
        process="u d~ > w+ h", kind="rambo", sqrt_s=500.0, masses=(0, 0, 80.4, 125.0), n=1 << 20, seed=9,
        cuts=None, s_ident=1.0,
        describe="u d~ > W+ H (s-channel W, WWH vertex), massive RAMBO at sqrt(s)=500 GeV, 2^20 points, seed 9"),
    "uux_wpwma": dict(
        process="u u~ > w+ w- a", kind="rambo", sqrt_s=500.0, masses=(0, 0, 80.4, 80.4, 0), n=1 << 20, seed=10,
        cuts=dict(legs=(4,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u u~ > W+ W- gamma (fifteen diagrams: the photon from the quark line and the W bosons, the "
                 "WWAA and WWAZ quartic vertices), massive RAMBO at sqrt(s)=500 GeV, photon pT>20, |eta|<2.5, "
                 "2^20 accepted points, seed 10"),
    "udx_wpg": dict(
        process="u d~ > w+ g", kind="rambo", sqrt_s=500.0, masses=(0, 0, 80.4, 0), n=1 << 20, seed=13,
        cuts=dict(legs=(3,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u d~ > W+ g (W plus one jet), massive RAMBO at sqrt(s)=500 GeV, gluon pT>20, |eta|<2.5, "
                 "2^20 accepted points, seed 13"),
    "uux_zg": dict(
        process="u u~ > z g", kind="rambo", sqrt_s=500.0, masses=(0, 0, 91.1876, 0), n=1 << 20, seed=14,
        cuts=dict(legs=(3,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u u~ > Z g (Z plus one jet), massive RAMBO at sqrt(s)=500 GeV, gluon pT>20, |eta|<2.5, "
                 "2^20 accepted points, seed 14"),
    "ug_wpd": dict(
        process="u g > w+ d", kind="rambo", sqrt_s=500.0, masses=(0, 0, 80.4, 0), n=1 << 20, seed=15,
        cuts=dict(legs=(3,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u g > W+ d (quark-gluon initial state), massive RAMBO at sqrt(s)=500 GeV, d-jet pT>20, "
                 "|eta|<2.5, 2^20 accepted points, seed 15"),
    "uux_zzg": dict(
        process="u u~ > z z g", kind="rambo", sqrt_s=500.0, masses=(0, 0, 91.1876, 91.1876, 0), n=1 << 20,
        seed=16, cuts=dict(legs=(4,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=0.5,
        describe="u u~ > Z Z g (Z pair plus one jet, six diagrams), massive RAMBO at sqrt(s)=500 GeV, gluon "
                 "pT>20, |eta|<2.5, 2^20 accepted points, seed 16"),
    "uux_zhg": dict(
        process="u u~ > z h g", kind="rambo", sqrt_s=600.0, masses=(0, 0, 91.1876, 125.0, 0), n=1 << 20, seed=18,
        cuts=dict(legs=(4,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u u~ > Z H g (Higgs-strahlung plus one jet), massive RAMBO at sqrt(s)=600 GeV, gluon pT>20, "
                 "|eta|<2.5, 2^20 accepted points, seed 18"),
    "udx_wphg": dict(
        process="u d~ > w+ h g", kind="rambo", sqrt_s=600.0, masses=(0, 0, 80.4, 125.0, 0), n=1 << 20, seed=23,
        cuts=dict(legs=(4,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u d~ > W+ H g (W Higgs-strahlung plus one jet), massive RAMBO at sqrt(s)=600 GeV, gluon pT>20, "
                 "|eta|<2.5, 2^20 accepted points, seed 23"),
    "udx_wpzg": dict(
        process="u d~ > w+ z g", kind="rambo", sqrt_s=600.0, masses=(0, 0, 80.4, 91.1876, 0), n=1 << 20, seed=19,
        cuts=dict(legs=(4,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u d~ > W+ Z g (W Z plus one jet, eight diagrams), massive RAMBO at sqrt(s)=600 GeV, gluon "
                 "pT>20, |eta|<2.5, 2^20 accepted points, seed 19"),
    "uux_wpwmg": dict(
        process="u u~ > w+ w- g", kind="rambo", sqrt_s=600.0, masses=(0, 0, 80.4, 80.4, 0), n=1 << 20, seed=20,
        cuts=dict(legs=(4,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u u~ > W+ W- g (W pair plus one jet, seven diagrams), massive RAMBO at sqrt(s)=600 GeV, gluon "
                 "pT>20, |eta|<2.5, 2^20 accepted points, seed 20"),
    "gg_wpdux": dict(
        process="g g > w+ d u~", kind="rambo", sqrt_s=600.0, masses=(0, 0, 80.4, 0, 0), n=1 << 20, seed=21,
        cuts=dict(legs=(3, 4), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=1.0,
        describe="g g > W+ d u~ (W plus two jets from two gluons, eight diagrams), massive RAMBO at sqrt(s)=600 "
                 "GeV, pT>20, |eta|<2.5, DeltaR>0.4 on the two quarks, 2^20 accepted points, seed 21"),
    "gg_zuux": dict(
        process="g g > z u u~", kind="rambo", sqrt_s=600.0, masses=(0, 0, 91.1876, 0, 0), n=1 << 20, seed=22,
        cuts=dict(legs=(3, 4), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=1.0,
        describe="g g > Z u u~ (Z plus two jets from two gluons, eight diagrams), massive RAMBO at sqrt(s)=600 "
                 "GeV, pT>20, |eta|<2.5, DeltaR>0.4 on the two quarks, 2^20 accepted points, seed 22"),
    "gg_ttx": dict(
        process="g g > t t~", kind="rambo", sqrt_s=800.0, masses=(0, 0, 175.0, 175.0), n=1 << 20, seed=11,
        cuts=None, s_ident=1.0,
        describe="g g > t t~ with on-shell tops (massive external spinors; t- and u-channel top exchange, "
                 "s-channel gluon), massive RAMBO at sqrt(s)=800 GeV, 2^20 points, seed 11"),
    "gg_ttxg": dict(
        process="g g > t t~ g", kind="rambo", sqrt_s=1000.0, masses=(0, 0, 175.0, 175.0, 0), n=1 << 20, seed=17,
        cuts=dict(legs=(4,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="g g > t t~ g (top pair plus one jet: sixteen diagrams with the three- and four-gluon "
                 "vertices), massive RAMBO at sqrt(s)=1 TeV, gluon pT>20, |eta|<2.5, 2^20 accepted points, "
                 "seed 17"),
    "uux_ttx": dict(
        process="u u~ > t t~", kind="rambo", sqrt_s=800.0, masses=(0, 0, 175.0, 175.0), n=1 << 20, seed=24,
        cuts=None, s_ident=1.0,
        describe="u u~ > t t~ with on-shell tops (s-channel gluon, photon and Z), massive RAMBO at sqrt(s)=800 "
                 "GeV, 2^20 points, seed 24"),
    "uux_ttxg": dict(
        process="u u~ > t t~ g", kind="rambo", sqrt_s=1000.0, masses=(0, 0, 175.0, 175.0, 0), n=1 << 20, seed=25,
        cuts=dict(legs=(4,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="u u~ > t t~ g (top pair plus one jet from q q~: thirteen diagrams with gluon, photon and Z "
                 "exchange), massive RAMBO at sqrt(s)=1 TeV, gluon pT>20, |eta|<2.5, 2^20 accepted points, seed 25"),
    "us_dch": dict(
        process="u s > d c h", kind="rambo", sqrt_s=1000.0, masses=(0, 0, 0, 0, 125.0), n=1 << 20, seed=26,
        cuts=None, s_ident=1.0,
        describe="u s > d c H (W+ W- fusion, one diagram), massive RAMBO at sqrt(s)=1 TeV, 2^20 points, seed 26"),
    "gg_ttxh": dict(
        process="g g > t t~ h", kind="rambo", sqrt_s=1000.0, masses=(0, 0, 175.0, 175.0, 125.0), n=1 << 20,
        seed=12, cuts=None, s_ident=1.0,
        describe="g g > t t~ H (eight diagrams: the Higgs from every top line through the FFS Yukawa vertex), "
                 "massive RAMBO at sqrt(s)=1 TeV, 2^20 points, seed 12"),
    "udx_wpgg": dict(
        process="u d~ > w+ g g", kind="rambo", sqrt_s=600.0, masses=(0, 0, 80.4, 0, 0), n=1 << 20, seed=41,
        cuts=dict(legs=(3, 4), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=0.5,
        describe="u d~ > W+ g g (on-shell W plus two jets, eight diagrams), massive RAMBO at sqrt(s)=600 GeV, "
                 "gluons pT>20, |eta|<2.5, DeltaR>0.4, 2^20 accepted points, seed 41"),
    "uux_zgg": dict(
        process="u u~ > z g g", kind="rambo", sqrt_s=600.0, masses=(0, 0, 91.1876, 0, 0), n=1 << 20, seed=42,
        cuts=dict(legs=(3, 4), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=0.5,
        describe="u u~ > Z g g (on-shell Z plus two jets, eight diagrams), massive RAMBO at sqrt(s)=600 GeV, "
                 "gluons pT>20, |eta|<2.5, DeltaR>0.4, 2^20 accepted points, seed 42"),
    "us_dchg": dict(
        process="u s > d c h g", kind="rambo", sqrt_s=1000.0, masses=(0, 0, 0, 0, 125.0, 0), n=1 << 20, seed=43,
        cuts=dict(legs=(2, 3, 5), pt_min=20.0, eta_max=5.0, dr_min=0.4), s_ident=1.0,
        describe="u s > d c H g (W+ W- fusion plus one jet, the gluon from either quark line), massive RAMBO at "
                 "sqrt(s)=1 TeV, the three jets pT>20, |eta|<5, DeltaR>0.4 (the gluon's collinear limits "
                 "with the outgoing quarks cut away), 2^20 accepted points, seed 43"),
    "us_dchhh": dict(
        process="u s > d c h h h", kind="rambo", sqrt_s=1500.0, masses=(0, 0, 0, 0, 125.0, 125.0, 125.0),
        n=1 << 20, seed=44, cuts=None, s_ident=1.0 / 6.0,
        describe="u s > d c H H H (W+ W- fusion into three Higgs bosons, 25 diagrams), massive RAMBO at "
                 "sqrt(s)=1.5 TeV, 2^20 points, seed 44"),
    "ud_udh": dict(
        process="u d > u d h", kind="rambo", sqrt_s=1000.0, masses=(0, 0, 0, 0, 125.0), n=1 << 20, seed=45,
        cuts=None, s_ident=1.0,
        describe="u d > u d H (Z Z and W+ W- fusion, interfering), massive RAMBO at sqrt(s)=1 TeV, 2^20 points, "
                 "seed 45"),
    "ud_udhh": dict(
        process="u d > u d h h", kind="rambo", sqrt_s=1000.0, masses=(0, 0, 0, 0, 125.0, 125.0), n=1 << 20,
        seed=46, cuts=None, s_ident=0.5,
        describe="u d > u d H H (Z Z and W+ W- fusion, eight diagrams), massive RAMBO at sqrt(s)=1 TeV, "
                 "2^20 points, seed 46"),
    "ud_udhhh": dict(
        process="u d > u d h h h", kind="rambo", sqrt_s=1500.0, masses=(0, 0, 0, 0, 125.0, 125.0, 125.0),
        n=1 << 20, seed=47, cuts=None, s_ident=1.0 / 6.0,
        describe="u d > u d H H H (the paper's Sect. 2.10 process: Z Z and W+ W- fusion, 50 diagrams), "
                 "massive RAMBO at sqrt(s)=1.5 TeV, 2^20 points, seed 47"),
    "ud_udhhh_cms": dict(
        process="u d > u d h h h", kind="rambo", sqrt_s=1500.0, masses=(0, 0, 0, 0, 125.0, 125.0, 125.0),
        n=1 << 20, seed=47, cuts=None, s_ident=1.0 / 6.0, params=dict(complex_mass=1),
        describe="u d > u d H H H with the complex-mass option of Sect. 7.11 (me_params.complex_mass = 1), "
                 "the same points as ud_udhhh"),
    "udx_wpggg": dict(
        process="u d~ > w+ g g g", kind="rambo", sqrt_s=800.0, masses=(0, 0, 80.4, 0, 0, 0), n=1 << 18, seed=48,
        cuts=dict(legs=(3, 4, 5), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=1.0 / 6.0,
        describe="u d~ > W+ g g g (on-shell W plus three jets, 54 diagrams, helicity-loop program), massive "
                 "RAMBO at sqrt(s)=800 GeV, gluons pT>20, |eta|<2.5, DeltaR>0.4, 2^18 accepted points, seed 48"),
    "gg_ttxhg": dict(
        process="g g > t t~ h g", kind="rambo", sqrt_s=1500.0, masses=(0, 0, 175.0, 175.0, 125.0, 0), n=1 << 18,
        seed=50, cuts=dict(legs=(5,), pt_min=20.0, eta_max=2.5, dr_min=0.0), s_ident=1.0,
        describe="g g > t t~ H g (H t t~ plus one jet, 54 diagrams, helicity-loop program), massive RAMBO at "
                 "sqrt(s)=1.5 TeV, gluon pT>20, |eta|<2.5, 2^18 accepted points, seed 50"),
    "us_dchgg": dict(
        process="u s > d c h g g", kind="rambo", sqrt_s=1000.0, masses=(0, 0, 0, 0, 125.0, 0, 0), n=1 << 20,
        seed=51, cuts=dict(legs=(2, 3, 5, 6), pt_min=20.0, eta_max=5.0, dr_min=0.4), s_ident=0.5,
        describe="u s > d c H g g (W+ W- fusion plus two jets, 24 diagrams), massive RAMBO at sqrt(s)=1 TeV, "
                 "the four jets pT>20, |eta|<5, DeltaR>0.4, 2^20 accepted points, seed 51"),
    "uux_zzgg": dict(
        process="u u~ > z z g g", kind="rambo", sqrt_s=600.0, masses=(0, 0, 91.1876, 91.1876, 0, 0), n=1 << 18,
        seed=52, cuts=dict(legs=(4, 5), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=0.25,
        describe="u u~ > Z Z g g (V V plus two jets, 30 diagrams, helicity-loop program), massive RAMBO at "
                 "sqrt(s)=600 GeV, gluons pT>20, |eta|<2.5, DeltaR>0.4, 2^18 accepted points, seed 52"),
    "uu_uuhh": dict(
        process="u u > u u h h", kind="rambo", sqrt_s=1000.0, masses=(0, 0, 0, 0, 125.0, 125.0), n=1 << 20,
        seed=54, cuts=None, s_ident=0.25,
        describe="u u > u u H H (Z Z fusion, identical quarks), massive RAMBO at sqrt(s)=1 TeV, 2^20 points, "
                 "seed 54"),
    "uu_uuhhh": dict(
        process="u u > u u h h h", kind="rambo", sqrt_s=1500.0, masses=(0, 0, 0, 0, 125.0, 125.0, 125.0),
        n=1 << 20, seed=55, cuts=None, s_ident=1.0 / 12.0,
        describe="u u > u u H H H (the paper's Sect. 2.10 process: Z Z fusion, identical quarks, 50 diagrams), "
                 "massive RAMBO at sqrt(s)=1.5 TeV, 2^20 points, seed 55"),
    "uux_wpwmgg": dict(
        process="u u~ > w+ w- g g", kind="rambo", sqrt_s=700.0, masses=(0, 0, 80.4, 80.4, 0, 0), n=1 << 18,
        seed=56, cuts=dict(legs=(4, 5), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=0.5,
        describe="u u~ > W+ W- g g (W+ W- plus two jets, 31 diagrams, helicity-loop program), massive RAMBO at "
                 "sqrt(s)=700 GeV, gluons pT>20, |eta|<2.5, DeltaR>0.4, 2^18 accepted points, seed 56"),
    "udx_wpzgg": dict(
        process="u d~ > w+ z g g", kind="rambo", sqrt_s=700.0, masses=(0, 0, 80.4, 91.1876, 0, 0), n=1 << 18,
        seed=57, cuts=dict(legs=(4, 5), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=0.5,
        describe="u d~ > W+ Z g g (W+ Z plus two jets, 38 diagrams, helicity-loop program), massive RAMBO at "
                 "sqrt(s)=700 GeV, gluons pT>20, |eta|<2.5, DeltaR>0.4, 2^18 accepted points, seed 57"),
    "udx_wphggg": dict(
        process="u d~ > w+ h g g g", kind="rambo", sqrt_s=900.0, masses=(0, 0, 80.4, 125.0, 0, 0, 0), n=1 << 18,
        seed=58, cuts=dict(legs=(4, 5, 6), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=1.0 / 6.0,
        describe="u d~ > W+ H g g g (H V plus three jets, 54 diagrams, helicity-loop program), massive RAMBO "
                 "at sqrt(s)=900 GeV, gluons pT>20, |eta|<2.5, DeltaR>0.4, 2^18 accepted points, seed 58"),
    "udx_wphgg": dict(
        process="u d~ > w+ h g g", kind="rambo", sqrt_s=700.0, masses=(0, 0, 80.4, 125.0, 0, 0), n=1 << 20,
        seed=53, cuts=dict(legs=(4, 5), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=0.5,
        describe="u d~ > W+ H g g (H V plus two jets, 8 diagrams), massive RAMBO at sqrt(s)=700 GeV, gluons "
                 "pT>20, |eta|<2.5, DeltaR>0.4, 2^20 accepted points, seed 53"),
    "uux_zggg": dict(
        process="u u~ > z g g g", kind="rambo", sqrt_s=800.0, masses=(0, 0, 91.1876, 0, 0, 0), n=1 << 18,
        seed=49, cuts=dict(legs=(3, 4, 5), pt_min=20.0, eta_max=2.5, dr_min=0.4), s_ident=1.0 / 6.0,
        describe="u u~ > Z g g g (on-shell Z plus three jets, 54 diagrams, helicity-loop program), massive "
                 "RAMBO at sqrt(s)=800 GeV, gluons pT>20, |eta|<2.5, DeltaR>0.4, 2^18 accepted points, seed 49"),
}

KIND = {"two_body": 0, "rambo": 1, "ttbar": 2, "rambo_bw": 3, "ypt": 4}

# The paper's selection, Eqs. 8-11: jets |eta| < 5, pT > 20 GeV and pT_ij = min(pT_i, pT_j) Delta R_ij
# > 20 GeV for every jet pair; b jets from top decays and charged leptons |eta| < 2.5, pT > 20 GeV
PAPER_CUTS = dict(jet_pt=20.0, jet_eta=5.0, jet_ptij=20.0, b_pt=20.0, b_eta=2.5, lep_pt=20.0, lep_eta=2.5)
JET, BJET, LEPTON = 1, 2, 3

# Workloads on the paper's own phase-space parametrisation (Eq. 13, App. A.1, Eq. 17, App. A.2) and
# selection (Eqs. 8-11), at the same partonic energies as the workloads above
PAPER_PS = {
    "udx_epvegg_ypt": dict(
        process="u d~ > e+ ve g g", kind="ypt", sqrt_s=1000.0, n=1 << 20, seed=31, s_ident=0.5,
        objects=[dict(legs=(4,), y_max=5.0, pt_min=20.0, pt_max=480.0),
                 dict(legs=(5,), y_max=5.0, pt_min=20.0, pt_max=480.0),
                 dict(legs=(2, 3), res_mass=80.4, res_width=2.085, y_max=5.0, pt_min=0.0, pt_max=480.0)],
        leg_class=(0, 0, LEPTON, 0, JET, JET),
        describe="u d~ > e+ ve g g at sqrt(s)=1 TeV on the paper's y, pT, phi parametrisation: the two "
                 "gluons and the W -> e+ ve resonance (Breit-Wigner, isotropic decay) as objects, pT "
                 "mapped by Eq. 17; the paper's cuts (jets |eta|<5, pT>20, pT_ij>20; lepton |eta|<2.5, "
                 "pT>20), 2^20 accepted points, seed 31"),
    "gg_gggg_ypt": dict(
        process="g g > g g g g", kind="ypt", sqrt_s=1500.0, n=1 << 18, seed=33, s_ident=1.0 / 24.0,
        objects=[dict(legs=(k,), y_max=5.0, pt_min=20.0, pt_max=700.0) for k in (2, 3, 4, 5)],
        leg_class=(0, 0, JET, JET, JET, JET),
        describe="g g > g g g g at sqrt(s)=1.5 TeV on the paper's y, pT, phi parametrisation with the "
                 "paper's jet cuts (|eta|<5, pT>20, pT_ij>20), 2^18 accepted points, seed 33"),
}


def kin_args(w):
    """Keyword arguments for binding.make_kin for a workload."""
    cut = w.get("cuts") or {}
    return dict(kind=KIND[w["kind"]], sqrt_s=w.get("sqrt_s", 0.0), sqrt_s_range=w.get("sqrt_s_range", (0.0, 0.0)),
                masses=w.get("masses", ()), cut_legs=cut.get("legs", ()), pt_min=cut.get("pt_min", 0.0),
                eta_max=cut.get("eta_max", 0.0), dr_min=cut.get("dr_min", 0.0), s_ident=w["s_ident"],
                res_mass=w.get("res_mass", 0.0), res_width=w.get("res_width", 0.0), objects=w.get("objects", ()),
                leg_class=w.get("leg_class"), paper_cuts=PAPER_CUTS if w.get("leg_class") else None)
