/*
 * FP64 CPU oracle for the HELIOS radiative-equilibrium hot path
 * (Malik et al. 2016, arXiv:1606.05474).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct
 * restatement of the paper's method in double precision.  It is used by the
 * tests, by the smoke check and by the CPU-baseline leg of the benchmark; no
 * product code path calls it.  It shares no code, header or table with the
 * CUDA library (include/helios.h and the package's csrc/).
 *
 * Units are CGS throughout (erg, cm, g, s, K); pressures enter in bar and are
 * converted to dyn cm^-2 (1 bar = 1e6) where the method needs them.
 *
 * Indexing convention (Sect. 2.2.1, Fig. 2): layer 0 is the bottom layer; the
 * BOA is interface 0 and the TOA is interface n.  With non-isothermal layers
 * every layer is split at its centre, giving 2n sublayers and 2n+1 points:
 * point 2i is interface i, point 2i+1 is the centre of layer i.  Sublayer s
 * lies between point s (below, "interface 1" of the paper's layer formulas)
 * and point s+1 (above, "interface 2").
 */
#ifndef HELIOS_REF_H
#define HELIOS_REF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n;                    /* layers */
    int L;                    /* wavelength bins used */
    int G;                    /* Gauss points per bin */
    double P_top_bar;         /* pressure of the top layer centre, bar */
    double P_bot_bar;         /* pressure of the bottom layer centre, bar */
    double grav;              /* surface gravity, cm s^-2 */
    double T_irr;             /* sigma*T_irr^4 = incident diffuse stellar flux */
    double T_int;             /* sigma*T_int^4 = internal heat flux */
    double T_star;            /* stellar blackbody temperature */
    const double* nu_edges;   /* [L+1] bin edges in cm^-1, increasing */
    const double* omega0;     /* [L] single-scattering albedo per bin */
    const double* g0;         /* [L] scattering asymmetry factor per bin */
    /* correlated-k table kappa[nP][nT][L_table][G], cm^2/g */
    int nP, nT, L_table;
    double log10P0, dlog10P;  /* pressure nodes log10P0 + k*dlog10P (bar) */
    double T0, dT;            /* temperature nodes T0 + k*dT (K) */
    const double* kappa;
    int grey;                 /* 1: two-band grey test mode (bin 0 visible, bin 1 thermal) */
    int rayleigh;             /* 1: H2 Rayleigh scattering (eqs. 16-17) added to every (sub)layer's
                                 opacity; omega0 per (sub)layer, point and g (the per-bin omega0 unused) */
} ref_atm;

typedef struct {
    double D;                 /* diffusivity factor (epsilon = 1/D) */
    double dtau_iso;          /* thin-sublayer switch to the isothermal form */
    double w0_pure;           /* pure-scattering switch on 1 - omega0 */
    double tol;               /* convergence threshold on |dF|/(sigma T^4) */
    double fpre_num;          /* f_pre numerator (1e5) */
    double fpre_exp;          /* f_pre exponent (0.9) */
    double osc_down;          /* timestep factor when oscillating (0.67) */
    double osc_up;            /* timestep factor when monotonic (1.1) */
    double mult_max;          /* cap on the timestep multiplier */
    double T_floor;           /* lower bound on temperature */
    double mbar_mp;           /* mean molecular mass in proton masses (2.4) */
    double n_dof;             /* degrees of freedom (5) */
    int n_scat;               /* additional scattering passes per temperature step (4) */
    int max_iter;             /* radiative-equilibrium iteration cap */
    int printed_gradient;     /* 1: use the gradient prefactor eps/(1+w0 g0) as printed */
    int tabulate;             /* 1: Planck and transmission functions from tables (Sect. 2.6) */
} ref_params;

enum { REF_CONVERGED = 0, REF_UPDATED = 1, REF_NOT_CONVERGED = 2, REF_NONFINITE = 3, REF_OUT_OF_RANGE = 4 };

void   ref_default_params(ref_params* p);

/* Tabulated functions of Sect. 2.6 (used by ref_flux_sweep when p->tabulate):
 * 1 - trans(x) on the nodes x_i = 10^(REF_TAB_X0 + 0.1 i), i < REF_TAB_NX, linear in x between
 * nodes (x below the first node: x itself; above the last: 1); the Planck intensity of bin l on
 * the nodes T_j = j REF_TAB_DT, j < REF_TAB_NT, linear in T (clamped to the end nodes). */
#define REF_TAB_X0 (-8.05)
#define REF_TAB_NX 102
#define REF_TAB_DT 10.0
#define REF_TAB_NT 601
double ref_tab_one_minus_trans(double x);
double ref_tab_planck_bin(double nu_lo, double nu_hi, double T);

/* special functions and quadrature */
double ref_E1(double x);
double ref_trans_exact(double dtau);            /* 2 E_3(dtau), eq. (6) */
double ref_diffusivity_exact(double dtau);      /* eq. (7) */
void   ref_gauss_legendre(int G, double* x, double* w);
double ref_planck_bin(double nu_lo, double nu_hi, double T);
double ref_rayleigh_kappa(double nu_lo, double nu_hi, double mbar_mp);

/* grid, temperatures at points, table lookup */
void   ref_grid(const ref_atm* a, double* log10P_pts, double* P_pts, double* dm_sub, double* P_lay);
void   ref_point_temperatures(int n, const double* T, double* T_pts);
void   ref_table_coord(double x, double x0, double dx, int nx, int* idx, double* w);
void   ref_interp_opacity(const ref_atm* a, const double* T, double* kappa_pts, int* idx_pts, double* w_pts);
void   ref_boundary_spectra(const ref_atm* a, double* toa, double* intern);

/* single-layer solutions */
void   ref_layer_twostream(double F1up, double F2dn, double B1, double B2, double dtau, double w0,
                           double g0, const ref_params* p, double* F2up, double* F1dn);
void   ref_layer_exact(double F1up, double F2dn, double B1, double B2, double dtau, double dtau_iso,
                       double* F2up, double* F1dn);

/* column sweeps and the radiative-equilibrium loop */
int    ref_flux_sweep(const ref_atm* a, const ref_params* p, const double* T, int n_passes, int exact,
                      double* warm, int warm_valid, double* Fup_bol, double* Fdn_bol, double* Fup_toa,
                      double* Fup_spec, double* Fdn_spec);
int    ref_flux_sweep_iso(const ref_atm* a, const ref_params* p, const double* T, int n_passes,
                          double* Fup_bol, double* Fdn_bol, double* Fup_toa);
void   ref_layer_affine(double B1, double B2, double dtau, double w0, double g0, const ref_params* p, double* c);
int    ref_flux_direct(const ref_atm* a, const ref_params* p, const double* T, int iso,
                       double* Fup_bol, double* Fdn_bol, double* Fup_toa);
int    ref_temp_update(const ref_atm* a, const ref_params* p, const double* Fup_bol, const double* Fdn_bol,
                       double* T, double* mult, int* hist, int* nhist, double* metric, double* dT);
int    ref_solve_re(const ref_atm* a, const ref_params* p, double* T, double* mult, int* hist, int* nhist,
                    double* warm, int* iters, double* metric);
int    ref_passes(const ref_atm* a, const ref_params* p);
/* host threads of the OpenMP loops over bins (for timing the oracle on 1 core and on all) */
void   ref_set_threads(int n);
int    ref_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
