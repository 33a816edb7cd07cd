"""Default cut constants of the Segment Linking chain (plain numbers).

The paper fixes only the 0.8 GeV stub threshold (Section 2); every other
constant is this project's reading. Both the device library and the oracle
receive the same values from here; neither derives them.
"""

DEFAULT_CUTS = dict(
    pt_min=0.8,            # GeV, stub / segment window threshold (Section 2)
    k_field=0.3,           # GeV / (T m)
    b_field=3.8,           # T
    z_lumi=20.0,           # cm, luminous region half length (3 sigma_z + 5 cm)
    n_md=3.0,              # MD window width in resolutions
    n_ls=3.0,              # LS windows
    n_t3=3.0,              # T3 beta and r-z windows
    n_t5=3.0,              # T5 inner/outer curvature consistency
    n_pt=3.0,              # pLS vs T3/T5 curvature consistency
    tol_r=0.05,            # |kappa| <= (1 + tol_r) / (pT_min radius)
    chi2_rphi_t5=15.0, chi2_rz_t5=17.0,
    chi2_rphi_pt3=17.0, chi2_rz_pt3=19.0,
    chi2_rphi_pt5=21.0, chi2_rz_pt5=23.0,
    pls_pt_tol=0.05,       # pLS keep pT >= pT_min (1 - tol)
    sig_pix=0.001,         # cm, pixel space-point resolution
    sb_eta_max=3.0, sb_n_eta=120, sb_n_phi=72,   # superbin binning (matches maps.MapParams)
    dr_clean=0.02,         # cross-cleaning eta-phi distance
    margin_rel=1e-5,       # relative margin of every threshold
)
