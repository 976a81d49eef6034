/*
 * FP64 CPU oracle for the HELIOS radiative-equilibrium hot path
 * (Malik et al. 2016, arXiv:1606.05474).
 *
 * TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
 * CPU-baseline leg of bench.py.  The CUDA library never calls it and shares
 * no code with it.  Build: gcc -O2 -ffp-contract=off -fopenmp (no FMA
 * contraction, so the table indices and weights follow IEEE double exactly).
 *
 * Each function states the passage of the paper it restates.  Where the paper
 * is silent, ambiguous or garbled, the reading taken is stated beside the code
 * with its justification.
 *
 * Parity pins: every function here is checked, in tests/test_oracle_*.py,
 * against something other than itself (library special functions, numerical
 * solution of the two-stream ODE, closed forms, invariants).  The
 * temperature-step oscillation rule (Sect. 2.2.4) is pinned against hand-made
 * sign sequences; the trajectory of the whole iteration is "parity unpinned"
 * (only its fixed point is pinned: net flux equals sigma*T_int^4 at
 * convergence).
 */
#include "helios_ref.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018, CGS */
static const double K_B = 1.380649e-16;          /* erg K^-1 */
static const double H_PL = 6.62607015e-27;       /* erg s */
static const double C_LIGHT = 2.99792458e10;     /* cm s^-1 */
static const double SIGMA_SB = 5.670374419e-5;   /* erg s^-1 cm^-2 K^-4 */
static const double M_PROTON = 1.67262192369e-24;/* g */
static const double PI = 3.14159265358979323846;
static const double EULER_GAMMA = 0.57721566490153286061;

void ref_default_params(ref_params* p)
{
    /* defaults: Sect. 3 (D = 2), Sect. 2.1.4 (1e-6), Sect. 2.2.1 (1e-4),
       Sect. 2.2.3 (4 extra scattering passes), Sect. 2.2.4 (1e5, 0.9, 33%,
       10%, 1e-7), Sect. 2.2.1 (mbar = 2.4 m_p), Sect. 2.2.3 (n_dof = 5) */
    p->D = 2.0;
    p->dtau_iso = 1e-4;
    p->w0_pure = 1e-6;
    p->tol = 1e-7;
    p->fpre_num = 1e5;
    p->fpre_exp = 0.9;
    p->osc_down = 0.67;
    p->osc_up = 1.1;
    p->mult_max = 10.0;
    p->T_floor = 1.0;
    p->mbar_mp = 2.4;
    p->n_dof = 5.0;
    p->n_scat = 4;
    p->max_iter = 20000;
    p->printed_gradient = 0;
    p->tabulate = 0;
}

/* ------------------------------------------------------------------------ */
/* Exponential integral E1 (needed by the exact transmission, eq. 6).
 * x <= 1: the power series of Abramowitz & Stegun 5.1.11,
 *   E1(x) = -gamma - ln x - sum_{k>=1} (-x)^k / (k k!).
 * x > 1: the continued fraction of A&S 5.1.22 in its even (contracted) form
 *   E1(x) = e^{-x} / (x+1 - 1^2/(x+3 - 2^2/(x+5 - ...))),
 * evaluated with the modified Lentz algorithm. */
double ref_E1(double x)
{
    if (x <= 0.0) return INFINITY;
    if (x <= 1.0) {
        double sum = 0.0, term = 1.0;
        for (int k = 1; k < 60; ++k) {
            term *= -x / k;                 /* (-x)^k / k! */
            double add = term / k;
            sum += add;
            if (fabs(add) < 1e-18 * fabs(sum)) break;
        }
        return -EULER_GAMMA - log(x) - sum;
    }
    const double tiny = 1e-300;
    double b = x + 1.0;
    double f = b, C = b, Dl = 0.0;
    for (int k = 1; k < 500; ++k) {
        double a = -(double)k * (double)k;
        b += 2.0;
        Dl = b + a * Dl;
        if (fabs(Dl) < tiny) Dl = tiny;
        C = b + a / C;
        if (fabs(C) < tiny) C = tiny;
        Dl = 1.0 / Dl;
        double delta = C * Dl;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-16) break;
    }
    return exp(-x) / f;
}

/* Exact flux transmission of a pure-absorbing slab, eq. (6):
 * T = 2 int_0^1 mu exp(-dtau/mu) dmu = (1 - dtau) e^{-dtau} + dtau^2 E1(dtau). */
double ref_trans_exact(double dtau)
{
    if (dtau <= 0.0) return 1.0;
    return (1.0 - dtau) * exp(-dtau) + dtau * dtau * ref_E1(dtau);
}

/* Exact diffusivity factor, eq. (7): D = -ln(T_exact)/dtau. */
double ref_diffusivity_exact(double dtau)
{
    return -log(ref_trans_exact(dtau)) / dtau;
}

/* Gauss-Legendre nodes and weights on [-1, 1], Sect. 2.3 eqs. (31)-(32):
 * y_g are the roots of P_G (Newton iteration on the three-term recurrence),
 * w_g = 2 / ((1 - y_g^2) P_G'(y_g)^2).  Returned in ascending order. */
void ref_gauss_legendre(int G, double* x, double* w)
{
    for (int i = 0; i < G; ++i) {
        double z = cos(PI * (i + 0.75) / (G + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < G; ++k) {
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_G(z), p0 = P_{G-1}(z) */
            dp = G * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < G; ++k) {
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = G * (z * p1 - p0) / (z * z - 1.0);
        }
        x[G - 1 - i] = z;                    /* cos guess runs high -> low */
        w[G - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (G == 1) { x[0] = 0.0; w[0] = 2.0; }
}

/* Planck intensity integrated over one wavenumber bin, evaluated at the bin
 * centre (Sect. 2.6: the Planck function at the model's wavelength values;
 * bins equal in wavenumber, Sect. 3):
 *   B_l(T) = 2 h c^2 nu_c^3 dnu / (exp(h c nu_c / (k T)) - 1),
 * in erg s^-1 cm^-2 sr^-1; pi*B_l is the bin's blackbody flux. */
double ref_planck_bin(double nu_lo, double nu_hi, double T)
{
    if (!(T > 0.0)) return 0.0;
    double nu = 0.5 * (nu_lo + nu_hi);
    double dnu = nu_hi - nu_lo;
    double x = H_PL * C_LIGHT * nu / (K_B * T);
    return 2.0 * H_PL * C_LIGHT * C_LIGHT * nu * nu * nu * dnu / expm1(x);
}

/* ------------------------------------------------------------------------ */
/* Opacity of Rayleigh scattering by H2 in a bin (Sect. 2.1.4): the cross section
 * sigma = 24 pi^3 / (n_ref^2 lambda^4) ((n^2 - 1)/(n^2 + 2))^2 K (eq. 16) with
 * n_ref = 2.68678e19 cm^-3, K = 1 and the refractive index
 * n = 13.58e-5 (1 + 7.52e-11 cm^2 / lambda^2) + 1 (eq. 17), at the bin's centre
 * wavelength lambda = 1/nu_c, divided by the mean molecular mass (cm^2/g). */
double ref_rayleigh_kappa(double nu_lo, double nu_hi, double mbar_mp)
{
    const double lam = 1.0 / (0.5 * (nu_lo + nu_hi));                      /* cm */
    const double n = 13.58e-5 * (1.0 + 7.52e-11 / (lam * lam)) + 1.0;
    const double f = (n * n - 1.0) / (n * n + 2.0);
    const double nref = 2.68678e19;
    const double sigma = 24.0 * PI * PI * PI / (nref * nref * pow(lam, 4)) * f * f;
    return sigma / (mbar_mp * M_PROTON);
}

/* Model grid, Sect. 2.2.1 and Fig. 2.  Layer centres are evenly spaced in
 * log10 P from P_bot (layer 0) to P_top (layer n-1); interfaces sit midway in
 * log P (the geometric mean of adjacent centres) and the outermost interfaces
 * half a step beyond the outermost centres.  Points: 2i interface i, 2i+1
 * centre of layer i.  Sublayer column mass dm_s = (P_s - P_{s+1}) / g,
 * eq. (19).  Output pressures in dyn cm^-2. */
void ref_grid(const ref_atm* a, double* log10P_pts, double* P_pts, double* dm_sub, double* P_lay)
{
    const int n = a->n;
    const double lb = log10(a->P_bot_bar), lt = log10(a->P_top_bar);
    const double h = (lb - lt) / (double)(n - 1);
    double* lp = log10P_pts;
    double* P = P_pts;
    double* tmpl = NULL;
    double* tmpP = NULL;
    if (!lp) lp = tmpl = (double*)malloc(sizeof(double) * (2 * n + 1));
    if (!P) P = tmpP = (double*)malloc(sizeof(double) * (2 * n + 1));
    for (int p = 0; p <= 2 * n; ++p) {
        lp[p] = (lb + 0.5 * h) - (0.5 * h) * (double)p;
        P[p] = 1e6 * pow(10.0, lp[p]);
    }
    if (dm_sub)
        for (int s = 0; s < 2 * n; ++s) dm_sub[s] = (P[s] - P[s + 1]) / a->grav;
    if (P_lay)
        for (int i = 0; i < n; ++i) P_lay[i] = P[2 * i + 1];
    free(tmpl);
    free(tmpP);
}

/* Temperatures at the 2n+1 points, Sect. 2.2.1: centres carry the layer
 * temperatures; interior interfaces are interpolated linearly in log P, which
 * on this grid (interface midway in log P) is the mean of the two centres.
 * Reading (the paper is silent): the BOA and TOA interfaces take the nearest
 * centre's temperature (no extrapolation). */
void ref_point_temperatures(int n, const double* T, double* T_pts)
{
    for (int i = 0; i < n; ++i) T_pts[2 * i + 1] = T[i];
    for (int i = 1; i < n; ++i) T_pts[2 * i] = 0.5 * (T[i - 1] + T[i]);
    T_pts[0] = T[0];
    T_pts[2 * n] = T[n - 1];
}

/* Index and weight of x on a uniform axis x0 + k*dx, k = 0..nx-1, for linear
 * interpolation (Sect. 2.3, last paragraphs and footnote): outside the table
 * the value of the nearest node is used, i.e. the weight is clamped to
 * [0, 1] with the index clamped to [0, nx-2]. */
void ref_table_coord(double x, double x0, double dx, int nx, int* idx, double* w)
{
    if (nx < 2) { *idx = 0; *w = 0.0; return; }
    double u = (x - x0) / dx;
    int i;
    if (!(u > 0.0)) i = 0;
    else if (u >= (double)(nx - 2)) i = nx - 2;
    else i = (int)floor(u);
    double t = (x - (x0 + (double)i * dx)) / dx;
    if (!(t > 0.0)) t = 0.0;
    if (t > 1.0) t = 1.0;
    *idx = i;
    *w = t;
}

static double table_value(const ref_atm* a, int iP, int iT, int l, int g)
{
    return a->kappa[(((size_t)iP * a->nT + iT) * a->L_table + l) * a->G + g];
}

/* Opacity at every point, bin and Gauss point (Sect. 2.3): the k-table is
 * interpolated bilinearly in (T, log10 P).  kappa_pts[p][l][g]; idx_pts[p] =
 * (iP, iT); w_pts[p] = (wP, wT). */
void ref_interp_opacity(const ref_atm* a, const double* T, double* kappa_pts, int* idx_pts, double* w_pts)
{
    const int n = a->n, np = 2 * n + 1;
    double* lp = (double*)malloc(sizeof(double) * np);
    double* Tp = (double*)malloc(sizeof(double) * np);
    ref_grid(a, lp, NULL, NULL, NULL);
    ref_point_temperatures(n, T, Tp);
    for (int p = 0; p < np; ++p) {
        int iP, iT;
        double wP, wT;
        ref_table_coord(lp[p], a->log10P0, a->dlog10P, a->nP, &iP, &wP);
        ref_table_coord(Tp[p], a->T0, a->dT, a->nT, &iT, &wT);
        if (idx_pts) { idx_pts[2 * p] = iP; idx_pts[2 * p + 1] = iT; }
        if (w_pts) { w_pts[2 * p] = wP; w_pts[2 * p + 1] = wT; }
        if (kappa_pts) {
            int iP1 = a->nP > 1 ? iP + 1 : iP, iT1 = a->nT > 1 ? iT + 1 : iT;
            for (int l = 0; l < a->L; ++l)
                for (int g = 0; g < a->G; ++g) {
                    double k00 = table_value(a, iP, iT, l, g), k10 = table_value(a, iP1, iT, l, g);
                    double k01 = table_value(a, iP, iT1, l, g), k11 = table_value(a, iP1, iT1, l, g);
                    kappa_pts[((size_t)p * a->L + l) * a->G + g] =
                        (1.0 - wT) * ((1.0 - wP) * k00 + wP * k10) + wT * ((1.0 - wP) * k01 + wP * k11);
                }
        }
    }
    free(lp);
    free(Tp);
}

/* Bin fluxes entering at the boundaries, Sect. 2.2.2 (eqs. 20-22).
 * TOA: the diffuse stellar flux f (R_star/a)^2 pi B_star; reading: T_irr^4
 * stands for f (R_star/a)^2 T_star^4, so the bins carry sigma*T_irr^4
 * distributed like a blackbody at T_star (the per-bin Planck values
 * normalised to sum to one).
 * BOA: the internal flux pi B_int = F0_up - F0_dn per bin, with
 * sum_l pi B_int,l = sigma*T_int^4, distributed like a blackbody at T_int.
 * Grey mode: bin 0 receives all stellar flux, bin 1 all internal flux. */
void ref_boundary_spectra(const ref_atm* a, double* toa, double* intern)
{
    const int L = a->L;
    if (a->grey) {
        for (int l = 0; l < L; ++l) toa[l] = intern[l] = 0.0;
        toa[0] = SIGMA_SB * pow(a->T_irr, 4);
        if (L > 1) intern[1] = SIGMA_SB * pow(a->T_int, 4);
        return;
    }
    double s_star = 0.0, s_int = 0.0;
    for (int l = 0; l < L; ++l) {
        s_star += ref_planck_bin(a->nu_edges[l], a->nu_edges[l + 1], a->T_star);
        s_int += ref_planck_bin(a->nu_edges[l], a->nu_edges[l + 1], a->T_int);
    }
    for (int l = 0; l < L; ++l) {
        double bs = ref_planck_bin(a->nu_edges[l], a->nu_edges[l + 1], a->T_star);
        double bi = ref_planck_bin(a->nu_edges[l], a->nu_edges[l + 1], a->T_int);
        toa[l] = (s_star > 0.0 && a->T_irr > 0.0) ? SIGMA_SB * pow(a->T_irr, 4) * bs / s_star : 0.0;
        intern[l] = (s_int > 0.0 && a->T_int > 0.0) ? SIGMA_SB * pow(a->T_int, 4) * bi / s_int : 0.0;
    }
}

/* Planck intensity of bin l at temperature T, or its grey-mode counterpart:
 * bin 0 (visible) does not emit, bin 1 (thermal) has pi*B = sigma*T^4. */
static double bin_planck(const ref_atm* a, int l, double T)
{
    if (a->grey) return l == 1 ? SIGMA_SB * pow(T, 4) / PI : 0.0;
    return ref_planck_bin(a->nu_edges[l], a->nu_edges[l + 1], T);
}

/* Sect. 2.6: "tabulate the Planck and the transmission functions" on a grid in T (10 K) and in
 * opacity (0.1 in log10).  Reading: the transmission of a layer is e^-x with x = lambda dtau
 * proportional to the layer's opacity, so a 0.1-dex grid in opacity is a 0.1-dex grid in x and
 * one table of x serves every layer and bin.  The table holds 1 - e^-x (exact where the layer
 * is thin) at the nodes x_i; between nodes it is linear in x. */
static double tab_node_x(int i) { return pow(10.0, REF_TAB_X0 + 0.1 * i); }

double ref_tab_one_minus_trans(double x)
{
    if (!(x > 0.0)) return 0.0;
    const int i = (int)floor((log10(x) - REF_TAB_X0) * 10.0);
    if (i < 0) return x;                       /* 1 - e^-x = x (1 + O(x)), x < 1e-8 */
    if (i >= REF_TAB_NX - 1) return 1.0;       /* e^-x < 1e-48 */
    const double x0 = tab_node_x(i), x1 = tab_node_x(i + 1);
    const double u0 = -expm1(-x0), u1 = -expm1(-x1);
    return u0 + (x - x0) / (x1 - x0) * (u1 - u0);
}

/* the Planck intensity of a bin, linear in T between the 10 K nodes (end nodes beyond) */
double ref_tab_planck_bin(double nu_lo, double nu_hi, double T)
{
    int j = (int)floor(T / REF_TAB_DT);
    if (j < 0) j = 0;
    if (j > REF_TAB_NT - 2) j = REF_TAB_NT - 2;
    double w = T / REF_TAB_DT - j;
    w = w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
    const double b0 = ref_planck_bin(nu_lo, nu_hi, j * REF_TAB_DT);
    const double b1 = ref_planck_bin(nu_lo, nu_hi, (j + 1) * REF_TAB_DT);
    return b0 + w * (b1 - b0);
}

/* ------------------------------------------------------------------------ */
/* Two-stream fluxes across one (sub)layer, Sect. 2.1.3, with eps = 1/D.
 * Inputs: upward flux entering from below (F1up), downward flux entering from
 * above (F2dn), Planck intensities at the lower (B1) and upper (B2) interface,
 * the optical thickness dtau > 0, omega0, g0.  Outputs F2up, F1dn.
 *
 *  - 1 - omega0 < w0_pure: pure-scattering form, eq. (14), tau0 = dtau.
 *  - dtau < dtau_iso: isothermal form with scattering, eqs. (11)-(13), with
 *    B = (B1 + B2)/2 (Sect. 2.2.1, last paragraph).
 *  - otherwise the non-isothermal form with scattering, eq. (15), with the
 *    transmission of eq. (8) and the coefficients of eqs. (12)-(13).
 *
 * Readings of eq. (15) (both fixed by solving the two-stream ODE whose
 * eigenvalue is eq. 8, whose coupling coefficients are eq. 13 and whose
 * thermal source reproduces eq. 9):
 *  - the emitted term of F2up carries B2 (the upper interface) with (alpha +
 *    beta) and B1 with xi, and symmetrically for F1dn; as printed the two
 *    Planck values are exchanged, which would make an optically thick layer
 *    emit its lower temperature from its top;
 *  - the gradient prefactor is eps/(1 - omega0 g0) (printed 1 + omega0 g0;
 *    they agree for g0 = 0), with B' = (B1 - B2)/dtau = dB/dtau, tau measured
 *    downwards (eq. 5). */
void ref_layer_twostream(double F1up, double F2dn, double B1, double B2, double dtau, double w0,
                         double g0, const ref_params* p, double* F2up, double* F1dn)
{
    const double D = p->D, eps = 1.0 / D;
    if (1.0 - w0 < p->w0_pure) {
        double a = D * (1.0 - g0) * dtau;
        double x = a * (F1up - F2dn) / (2.0 + a);
        *F2up = F1up - x;
        *F1dn = F2dn + x;
        return;
    }
    const double x = D * sqrt((1.0 - w0 * g0) * (1.0 - w0)) * dtau;
    double trans = p->tabulate ? 1.0 - ref_tab_one_minus_trans(x) : exp(-x);    /* eq. (8) */
    double r = sqrt((1.0 - w0) / (1.0 - w0 * g0));
    double zp = 0.5 * (1.0 + r), zm = 0.5 * (1.0 - r);                          /* eq. (13) */
    double alpha = zm * zm * trans * trans - zp * zp;                           /* eq. (12) */
    double beta = zp * zm * (1.0 - trans * trans);
    double xi = (zm * zm - zp * zp) * trans;
    if (dtau < p->dtau_iso) {
        double ups = (zm * zm * trans + zp * zp) * (1.0 - trans);
        double B = 0.5 * (B1 + B2);
        *F2up = (xi * F1up - beta * F2dn + 2.0 * PI * eps * B * (beta - ups)) / alpha;  /* eq. (11) */
        *F1dn = (xi * F2dn - beta * F1up + 2.0 * PI * eps * B * (beta - ups)) / alpha;
        return;
    }
    double Bp = (B1 - B2) / dtau;                                               /* eq. (5) */
    double c = eps * Bp / (p->printed_gradient ? (1.0 + w0 * g0) : (1.0 - w0 * g0));
    *F2up = (xi * F1up - beta * F2dn
             + 2.0 * PI * eps * (B2 * (alpha + beta) - B1 * xi + c * (alpha - xi - beta))) / alpha;
    *F1dn = (xi * F2dn - beta * F1up
             + 2.0 * PI * eps * (B1 * (alpha + beta) - B2 * xi + c * (xi - alpha + beta))) / alpha;
}

/* Exact pure-absorption solution across one layer (no two-stream closure),
 * Sect. 2.1.2: isothermal eq. (3) (B = (B1+B2)/2 below dtau_iso) and linear-B
 * eq. (4), with the exact transmission of eq. (6).  Reading of eq. (4):
 * dtau > 0 is the layer's optical thickness and B' = (B1 - B2)/dtau with
 * interface 1 below interface 2; with that reading eq. (4) is exactly the
 * angular integral of the formal solution for B linear in tau. */
void ref_layer_exact(double F1up, double F2dn, double B1, double B2, double dtau, double dtau_iso,
                     double* F2up, double* F1dn)
{
    double tr = ref_trans_exact(dtau);
    if (dtau < dtau_iso) {
        double B = 0.5 * (B1 + B2);
        *F2up = tr * F1up + PI * B * (1.0 - tr);
        *F1dn = tr * F2dn + PI * B * (1.0 - tr);
        return;
    }
    double Bp = (B1 - B2) / dtau;
    double grad = (2.0 / 3.0) * (1.0 - exp(-dtau)) - dtau * (1.0 - tr / 3.0);
    *F2up = tr * F1up + PI * B1 * (1.0 - tr) + PI * Bp * grad;
    *F1dn = tr * F2dn + PI * B2 * (1.0 - tr) - PI * Bp * grad;
}

/* Number of flux passes per temperature step (Sect. 2.2.3): one plus the
 * additional scattering passes when any bin scatters; one otherwise (with
 * omega0 = 0 the up and down streams decouple and one pass is exact). */
void ref_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int ref_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int ref_passes(const ref_atm* a, const ref_params* p)
{
    if (a->rayleigh) return 1 + p->n_scat;
    for (int l = 0; l < a->L; ++l)
        if (a->omega0[l] != 0.0) return 1 + p->n_scat;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* One flux evaluation of the whole column for every bin and Gauss point.
 *
 * Per (bin l, Gauss point g): opacity at the points (Sect. 2.3), sublayer
 * opacity = mean of its two end points (Sect. 2.3), dtau_s = kappa_s dm_s
 * (eq. 19); then n_passes passes, each a downward sweep from the TOA
 * (F_2n,dn = TOA_l, eq. 20) using the upward fluxes of the previous pass,
 * the BOA condition F0_up = F0_dn + pi B_int,l (eq. 22), and an upward sweep
 * using the downward fluxes just computed (Sect. 2.2.3: the coupled streams
 * start from zero and are refined in place; later temperature steps start
 * from the previous step's upward fluxes when warm != NULL && warm_valid).
 *
 * Gauss-point sum (Sect. 2.3, eqs. 30-33): F_l = sum_g (w_g/2) F_g with the
 * Gauss-Legendre weights of [-1, 1] (reading: eq. 33 omits the factor 1/2 of
 * eq. 31; the weights on [0, 1] are w_g/2 and sum to one).  Bolometric
 * fluxes (Sect. 2.2.3) are the sums over bins at the interfaces.
 *
 * exact != 0: pure absorption with the exact layer solution (eqs. 3-6), one
 * pass.  warm: [L][G][2n+1] upward fluxes, in/out.  Fup_bol/Fdn_bol: [n+1].
 * Fup_toa: [L] emergent spectrum.  Fup_spec/Fdn_spec: [L][2n+1] bin fluxes
 * at every point (optional).  Returns 0, or -1 on a non-finite flux. */
int ref_flux_sweep(const ref_atm* a, const ref_params* p, const double* T, int n_passes, int exact,
                   double* warm, int warm_valid, double* Fup_bol, double* Fdn_bol, double* Fup_toa,
                   double* Fup_spec, double* Fdn_spec)
{
    const int n = a->n, np = 2 * n + 1, L = a->L, G = a->G;
    double* lp = (double*)malloc(sizeof(double) * np);
    double* dm = (double*)malloc(sizeof(double) * (np - 1));
    double* Tp = (double*)malloc(sizeof(double) * np);
    double* gx = (double*)malloc(sizeof(double) * G);
    double* gw = (double*)malloc(sizeof(double) * G);
    double* toa = (double*)malloc(sizeof(double) * L);
    double* bint = (double*)malloc(sizeof(double) * L);
    int* iP = (int*)malloc(sizeof(int) * np);
    int* iT = (int*)malloc(sizeof(int) * np);
    double* wP = (double*)malloc(sizeof(double) * np);
    double* wT = (double*)malloc(sizeof(double) * np);
    double* up_bin = (double*)calloc((size_t)L * (n + 1), sizeof(double));
    double* dn_bin = (double*)calloc((size_t)L * (n + 1), sizeof(double));
    int bad = 0;

    ref_grid(a, lp, NULL, dm, NULL);
    ref_point_temperatures(n, T, Tp);
    ref_gauss_legendre(G, gx, gw);
    ref_boundary_spectra(a, toa, bint);
    for (int q = 0; q < np; ++q) {
        ref_table_coord(lp[q], a->log10P0, a->dlog10P, a->nP, &iP[q], &wP[q]);
        ref_table_coord(Tp[q], a->T0, a->dT, a->nT, &iT[q], &wT[q]);
    }
    if (exact) n_passes = 1;

#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (int l = 0; l < L; ++l) {
        double* B = (double*)malloc(sizeof(double) * np);
        double* kap = (double*)malloc(sizeof(double) * np);
        double* dtau = (double*)malloc(sizeof(double) * (np - 1));
        double* Fup = (double*)malloc(sizeof(double) * np);
        double* Fdn = (double*)malloc(sizeof(double) * np);
        const double g0 = a->g0[l];
        const double kR = a->rayleigh ? ref_rayleigh_kappa(a->nu_edges[l], a->nu_edges[l + 1], p->mbar_mp) : 0.0;
        double* w0s = (double*)malloc(sizeof(double) * (np - 1));
        for (int q = 0; q < np; ++q)
            B[q] = (p->tabulate && !a->grey) ? ref_tab_planck_bin(a->nu_edges[l], a->nu_edges[l + 1], Tp[q])
                                             : bin_planck(a, l, Tp[q]);
        if (Fup_spec) memset(Fup_spec + (size_t)l * np, 0, sizeof(double) * np);
        if (Fdn_spec) memset(Fdn_spec + (size_t)l * np, 0, sizeof(double) * np);
        if (Fup_toa) Fup_toa[l] = 0.0;
        for (int g = 0; g < G; ++g) {
            const double wg = 0.5 * gw[g];
            for (int q = 0; q < np; ++q) {
                int i1 = a->nP > 1 ? iP[q] + 1 : iP[q], j1 = a->nT > 1 ? iT[q] + 1 : iT[q];
                double k00 = table_value(a, iP[q], iT[q], l, g), k10 = table_value(a, i1, iT[q], l, g);
                double k01 = table_value(a, iP[q], j1, l, g), k11 = table_value(a, i1, j1, l, g);
                kap[q] = (1.0 - wT[q]) * ((1.0 - wP[q]) * k00 + wP[q] * k10)
                       + wT[q] * ((1.0 - wP[q]) * k01 + wP[q] * k11);
            }
            /* sublayer opacity: the mean of its end points (Sect. 2.3), plus the Rayleigh
             * opacity, whose share of it is the sublayer's omega0 (Sect. 2.1.4) */
            for (int s = 0; s < np - 1; ++s) {
                const double kabs = 0.5 * (kap[s] + kap[s + 1]);
                dtau[s] = (kabs + kR) * dm[s];
                w0s[s] = a->rayleigh ? kR / (kabs + kR) : a->omega0[l];
            }
            double* wcol = warm ? warm + ((size_t)l * G + g) * np : NULL;
            for (int q = 0; q < np; ++q) Fup[q] = (wcol && warm_valid) ? wcol[q] : 0.0;
            for (int pass = 0; pass < n_passes; ++pass) {
                double up_dummy, dn_dummy;
                Fdn[np - 1] = toa[l];
                for (int s = np - 2; s >= 0; --s) {
                    if (exact)
                        ref_layer_exact(Fup[s], Fdn[s + 1], B[s], B[s + 1], dtau[s], p->dtau_iso, &up_dummy, &Fdn[s]);
                    else
                        ref_layer_twostream(Fup[s], Fdn[s + 1], B[s], B[s + 1], dtau[s], w0s[s], g0, p, &up_dummy,
                                            &Fdn[s]);
                }
                Fup[0] = Fdn[0] + bint[l];
                for (int s = 0; s < np - 1; ++s) {
                    if (exact)
                        ref_layer_exact(Fup[s], Fdn[s + 1], B[s], B[s + 1], dtau[s], p->dtau_iso, &Fup[s + 1], &dn_dummy);
                    else
                        ref_layer_twostream(Fup[s], Fdn[s + 1], B[s], B[s + 1], dtau[s], w0s[s], g0, p, &Fup[s + 1],
                                            &dn_dummy);
                }
            }
            if (wcol) memcpy(wcol, Fup, sizeof(double) * np);
            for (int i = 0; i <= n; ++i) {
                up_bin[(size_t)l * (n + 1) + i] += wg * Fup[2 * i];
                dn_bin[(size_t)l * (n + 1) + i] += wg * Fdn[2 * i];
            }
            if (Fup_toa) Fup_toa[l] += wg * Fup[np - 1];
            if (Fup_spec) for (int q = 0; q < np; ++q) Fup_spec[(size_t)l * np + q] += wg * Fup[q];
            if (Fdn_spec) for (int q = 0; q < np; ++q) Fdn_spec[(size_t)l * np + q] += wg * Fdn[q];
            for (int q = 0; q < np; ++q)
                if (!isfinite(Fup[q]) || !isfinite(Fdn[q])) bad = 1;
        }
        free(B); free(kap); free(dtau); free(Fup); free(Fdn); free(w0s);
    }
    for (int i = 0; i <= n; ++i) {
        double su = 0.0, sd = 0.0;
        for (int l = 0; l < L; ++l) {
            su += up_bin[(size_t)l * (n + 1) + i];
            sd += dn_bin[(size_t)l * (n + 1) + i];
        }
        Fup_bol[i] = su;
        Fdn_bol[i] = sd;
    }
    free(lp); free(dm); free(Tp); free(gx); free(gw); free(toa); free(bint);
    free(iP); free(iT); free(wP); free(wT); free(up_bin); free(dn_bin);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Two-stream fluxes across one isothermal layer of Planck intensity B,
 * Sect. 2.1.3: eq. (9) without scattering (omega0 = 0), eq. (11) with the
 * coefficients of eq. (12) and the coupling coefficients of eq. (13) otherwise,
 * and the pure-scattering form eq. (14) when 1 - omega0 < w0_pure.  Inputs and
 * outputs as ref_layer_twostream. */
static void iso_layer(double F1up, double F2dn, double B, double dtau, double w0, double g0,
                      const ref_params* p, double* F2up, double* F1dn)
{
    const double D = p->D, eps = 1.0 / D;
    if (1.0 - w0 < p->w0_pure) {
        double a = D * (1.0 - g0) * dtau;
        double x = a * (F1up - F2dn) / (2.0 + a);
        *F2up = F1up - x;
        *F1dn = F2dn + x;
        return;
    }
    double trans = exp(-D * sqrt((1.0 - w0 * g0) * (1.0 - w0)) * dtau);        /* eq. (8) */
    if (w0 == 0.0) {                                                            /* eq. (9) */
        *F2up = trans * F1up + 2.0 * PI * eps * B * (1.0 - trans);
        *F1dn = trans * F2dn + 2.0 * PI * eps * B * (1.0 - trans);
        return;
    }
    double r = sqrt((1.0 - w0) / (1.0 - w0 * g0));
    double zp = 0.5 * (1.0 + r), zm = 0.5 * (1.0 - r);                          /* eq. (13) */
    double alpha = zm * zm * trans * trans - zp * zp;                           /* eq. (12) */
    double beta = zp * zm * (1.0 - trans * trans);
    double xi = (zm * zm - zp * zp) * trans;
    double ups = (zm * zm * trans + zp * zp) * (1.0 - trans);
    *F2up = (xi * F1up - beta * F2dn + 2.0 * PI * eps * B * (beta - ups)) / alpha;   /* eq. (11) */
    *F1dn = (xi * F2dn - beta * F1up + 2.0 * PI * eps * B * (beta - ups)) / alpha;
}

/* One flux evaluation on the grid of isothermal layers (Sect. 2.2.1, first
 * part), the grid of the emission spectra computed after convergence (Sect. 3:
 * a post-processing step).  Layer i has the temperature T[i] and the pressure
 * of its centre (the same centres as the non-isothermal grid), its opacity is
 * interpolated there (Sect. 2.3), and its optical thickness is kappa_i dm_i with
 * dm_i = (P_i - P_{i+1})/g between its interfaces (eq. 19).  Layer fluxes from
 * eqs. (9), (11) or (14) with B_i = B(T_i).  Passes, boundary conditions (eqs.
 * 20, 22) and the Gauss-point and bin sums as ref_flux_sweep, each pass from
 * the previous pass's upward fluxes, the first from zero.  Fup_bol, Fdn_bol:
 * [n+1] at the interfaces; Fup_toa: [L] (optional).  Returns 0, or -1 on a
 * non-finite flux. */
int ref_flux_sweep_iso(const ref_atm* a, const ref_params* p, const double* T, int n_passes,
                       double* Fup_bol, double* Fdn_bol, double* Fup_toa)
{
    const int n = a->n, np = 2 * n + 1, L = a->L, G = a->G;
    double* lp = (double*)malloc(sizeof(double) * np);
    double* Pp = (double*)malloc(sizeof(double) * np);
    double* gx = (double*)malloc(sizeof(double) * G);
    double* gw = (double*)malloc(sizeof(double) * G);
    double* toa = (double*)malloc(sizeof(double) * L);
    double* bint = (double*)malloc(sizeof(double) * L);
    double* dm = (double*)malloc(sizeof(double) * n);
    int* iP = (int*)malloc(sizeof(int) * n);
    int* iT = (int*)malloc(sizeof(int) * n);
    double* wP = (double*)malloc(sizeof(double) * n);
    double* wT = (double*)malloc(sizeof(double) * n);
    double* up_bin = (double*)calloc((size_t)L * (n + 1), sizeof(double));
    double* dn_bin = (double*)calloc((size_t)L * (n + 1), sizeof(double));
    int bad = 0;

    ref_grid(a, lp, Pp, NULL, NULL);              /* points 2i: interfaces, 2i+1: centres */
    ref_gauss_legendre(G, gx, gw);
    ref_boundary_spectra(a, toa, bint);
    for (int i = 0; i < n; ++i) {
        dm[i] = (Pp[2 * i] - Pp[2 * i + 2]) / a->grav;
        ref_table_coord(lp[2 * i + 1], a->log10P0, a->dlog10P, a->nP, &iP[i], &wP[i]);
        ref_table_coord(T[i], a->T0, a->dT, a->nT, &iT[i], &wT[i]);
    }

#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (int l = 0; l < L; ++l) {
        double* B = (double*)malloc(sizeof(double) * n);
        double* dtau = (double*)malloc(sizeof(double) * n);
        double* Fup = (double*)malloc(sizeof(double) * (n + 1));
        double* Fdn = (double*)malloc(sizeof(double) * (n + 1));
        const double g0 = a->g0[l];
        const double kR = a->rayleigh ? ref_rayleigh_kappa(a->nu_edges[l], a->nu_edges[l + 1], p->mbar_mp) : 0.0;
        double* w0s = (double*)malloc(sizeof(double) * n);
        for (int i = 0; i < n; ++i) B[i] = bin_planck(a, l, T[i]);
        if (Fup_toa) Fup_toa[l] = 0.0;
        for (int g = 0; g < G; ++g) {
            const double wg = 0.5 * gw[g];
            for (int i = 0; i < n; ++i) {
                int i1 = a->nP > 1 ? iP[i] + 1 : iP[i], j1 = a->nT > 1 ? iT[i] + 1 : iT[i];
                double k00 = table_value(a, iP[i], iT[i], l, g), k10 = table_value(a, i1, iT[i], l, g);
                double k01 = table_value(a, iP[i], j1, l, g), k11 = table_value(a, i1, j1, l, g);
                double kap = (1.0 - wT[i]) * ((1.0 - wP[i]) * k00 + wP[i] * k10)
                           + wT[i] * ((1.0 - wP[i]) * k01 + wP[i] * k11);
                dtau[i] = (kap + kR) * dm[i];                      /* Rayleigh opacity, Sect. 2.1.4 */
                w0s[i] = a->rayleigh ? kR / (kap + kR) : a->omega0[l];
            }
            for (int i = 0; i <= n; ++i) Fup[i] = 0.0;
            for (int pass = 0; pass < n_passes; ++pass) {
                double dummy;
                Fdn[n] = toa[l];
                for (int i = n - 1; i >= 0; --i)
                    iso_layer(Fup[i], Fdn[i + 1], B[i], dtau[i], w0s[i], g0, p, &dummy, &Fdn[i]);
                Fup[0] = Fdn[0] + bint[l];
                for (int i = 0; i < n; ++i)
                    iso_layer(Fup[i], Fdn[i + 1], B[i], dtau[i], w0s[i], g0, p, &Fup[i + 1], &dummy);
            }
            for (int i = 0; i <= n; ++i) {
                up_bin[(size_t)l * (n + 1) + i] += wg * Fup[i];
                dn_bin[(size_t)l * (n + 1) + i] += wg * Fdn[i];
                if (!isfinite(Fup[i]) || !isfinite(Fdn[i])) bad = 1;
            }
            if (Fup_toa) Fup_toa[l] += wg * Fup[n];
        }
        free(B); free(dtau); free(Fup); free(Fdn); free(w0s);
    }
    for (int i = 0; i <= n; ++i) {
        double su = 0.0, sd = 0.0;
        for (int l = 0; l < L; ++l) {
            su += up_bin[(size_t)l * (n + 1) + i];
            sd += dn_bin[(size_t)l * (n + 1) + i];
        }
        Fup_bol[i] = su;
        Fdn_bol[i] = sd;
    }
    free(lp); free(Pp); free(gx); free(gw); free(toa); free(bint); free(dm);
    free(iP); free(iT); free(wP); free(wT); free(up_bin); free(dn_bin);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* The layer solutions of Sect. 2.1.3 are affine in the incoming fluxes:
 *     F2up = c[0] F1up + c[1] F2dn + c[2],   F1dn = c[3] F2dn + c[4] F1up + c[5].
 * ref_layer_affine returns the six coefficients of ref_layer_twostream's layer
 * (eq. 14 for pure scattering, eq. 11 below dtau_iso, else eq. 15, with the same
 * readings); iso_affine those of an isothermal layer of Planck intensity B
 * (eq. 9 without scattering, eq. 11 with it, eq. 14 for pure scattering). */
void ref_layer_affine(double B1, double B2, double dtau, double w0, double g0, const ref_params* p, double* c)
{
    const double D = p->D, eps = 1.0 / D;
    if (1.0 - w0 < p->w0_pure) {                                                /* eq. (14) */
        double a = D * (1.0 - g0) * dtau;
        c[0] = c[3] = 2.0 / (2.0 + a);
        c[1] = c[4] = a / (2.0 + a);
        c[2] = c[5] = 0.0;
        return;
    }
    double trans = exp(-D * sqrt((1.0 - w0 * g0) * (1.0 - w0)) * dtau);        /* eq. (8) */
    double r = sqrt((1.0 - w0) / (1.0 - w0 * g0));
    double zp = 0.5 * (1.0 + r), zm = 0.5 * (1.0 - r);                          /* eq. (13) */
    double alpha = zm * zm * trans * trans - zp * zp;                           /* eq. (12) */
    double beta = zp * zm * (1.0 - trans * trans);
    double xi = (zm * zm - zp * zp) * trans;
    c[0] = c[3] = xi / alpha;
    c[1] = c[4] = -beta / alpha;
    if (dtau < p->dtau_iso) {                                                   /* eq. (11) */
        double ups = (zm * zm * trans + zp * zp) * (1.0 - trans);
        double B = 0.5 * (B1 + B2);
        c[2] = c[5] = 2.0 * PI * eps * B * (beta - ups) / alpha;
        return;
    }
    double Bp = (B1 - B2) / dtau;                                               /* eq. (15) */
    double g = eps * Bp / (p->printed_gradient ? (1.0 + w0 * g0) : (1.0 - w0 * g0));
    c[2] = 2.0 * PI * eps * (B2 * (alpha + beta) - B1 * xi + g * (alpha - xi - beta)) / alpha;
    c[5] = 2.0 * PI * eps * (B1 * (alpha + beta) - B2 * xi + g * (xi - alpha + beta)) / alpha;
}

static void iso_affine(double B, double dtau, double w0, double g0, const ref_params* p, double* c)
{
    const double D = p->D, eps = 1.0 / D;
    if (1.0 - w0 < p->w0_pure) {                                                /* eq. (14) */
        double a = D * (1.0 - g0) * dtau;
        c[0] = c[3] = 2.0 / (2.0 + a);
        c[1] = c[4] = a / (2.0 + a);
        c[2] = c[5] = 0.0;
        return;
    }
    double trans = exp(-D * sqrt((1.0 - w0 * g0) * (1.0 - w0)) * dtau);        /* eq. (8) */
    if (w0 == 0.0) {                                                            /* eq. (9) */
        c[0] = c[3] = trans;
        c[1] = c[4] = 0.0;
        c[2] = c[5] = 2.0 * PI * eps * B * (1.0 - trans);
        return;
    }
    double r = sqrt((1.0 - w0) / (1.0 - w0 * g0));
    double zp = 0.5 * (1.0 + r), zm = 0.5 * (1.0 - r);
    double alpha = zm * zm * trans * trans - zp * zp;
    double beta = zp * zm * (1.0 - trans * trans);
    double xi = (zm * zm - zp * zp) * trans;
    double ups = (zm * zm * trans + zp * zp) * (1.0 - trans);
    c[0] = c[3] = xi / alpha;                                                   /* eq. (11) */
    c[1] = c[4] = -beta / alpha;
    c[2] = c[5] = 2.0 * PI * eps * B * (beta - ups) / alpha;
}

/* Solve A x = b for a square matrix whose nonzeros lie within kl sub- and ku
 * super-diagonals: Gaussian elimination with partial pivoting, the loops limited
 * to the band (pivoting widens the upper band to ku + kl).  A is dense, row-major,
 * overwritten; x returned in b.  Returns -1 on a zero pivot. */
static int band_solve(int N, int kl, int ku, double* A, double* b)
{
    for (int j = 0; j < N; ++j) {
        int piv = j;
        int last = j + kl < N - 1 ? j + kl : N - 1;
        for (int i = j + 1; i <= last; ++i)
            if (fabs(A[(size_t)i * N + j]) > fabs(A[(size_t)piv * N + j])) piv = i;
        if (A[(size_t)piv * N + j] == 0.0) return -1;
        int cmax = j + ku + kl < N - 1 ? j + ku + kl : N - 1;
        if (piv != j) {
            for (int k = j; k <= cmax; ++k) {
                double t = A[(size_t)j * N + k]; A[(size_t)j * N + k] = A[(size_t)piv * N + k]; A[(size_t)piv * N + k] = t;
            }
            double t = b[j]; b[j] = b[piv]; b[piv] = t;
        }
        for (int i = j + 1; i <= last; ++i) {
            double f = A[(size_t)i * N + j] / A[(size_t)j * N + j];
            if (f == 0.0) continue;
            for (int k = j; k <= cmax; ++k) A[(size_t)i * N + k] -= f * A[(size_t)j * N + k];
            b[i] -= f * b[j];
        }
    }
    for (int j = N - 1; j >= 0; --j) {
        int cmax = j + ku + kl < N - 1 ? j + ku + kl : N - 1;
        double s = b[j];
        for (int k = j + 1; k <= cmax; ++k) s -= A[(size_t)j * N + k] * b[k];
        b[j] = s / A[(size_t)j * N + j];
    }
    return 0;
}

/* The exact solution of the coupled two-stream equations of every column: the
 * limit that the scattering passes of Sect. 2.2.3 approach (each pass is one
 * sweep of a block Gauss-Seidel iteration on this system).  Per (bin, g) the
 * unknowns are the upward and downward fluxes at the N points of the column
 * (x[2k] = F_up,k, x[2k+1] = F_dn,k); the equations are the BOA condition
 * F_up,0 - F_dn,0 = pi B_int (eq. 22), the two layer equations of every
 * (sub)layer in affine form, and the TOA condition F_dn,N-1 = TOA (eq. 20);
 * solved by banded Gaussian elimination.  iso = 0: the sublayered grid of
 * ref_flux_sweep; iso = 1: the isothermal-layer grid of ref_flux_sweep_iso.
 * Outputs as those functions.  Returns 0, or -1 on a non-finite flux or a
 * singular system. */
int ref_flux_direct(const ref_atm* a, const ref_params* p, const double* T, int iso,
                    double* Fup_bol, double* Fdn_bol, double* Fup_toa)
{
    const int n = a->n, L = a->L, G = a->G, np = 2 * n + 1;
    const int N = iso ? n + 1 : np;               /* points of a column */
    double* lp = (double*)malloc(sizeof(double) * np);
    double* Pp = (double*)malloc(sizeof(double) * np);
    double* dm = (double*)malloc(sizeof(double) * (np - 1));
    double* Tq = (double*)malloc(sizeof(double) * np);
    double* gx = (double*)malloc(sizeof(double) * G);
    double* gw = (double*)malloc(sizeof(double) * G);
    double* toa = (double*)malloc(sizeof(double) * L);
    double* bint = (double*)malloc(sizeof(double) * L);
    int* iP = (int*)malloc(sizeof(int) * np);
    int* iT = (int*)malloc(sizeof(int) * np);
    double* wP = (double*)malloc(sizeof(double) * np);
    double* wT = (double*)malloc(sizeof(double) * np);
    double* dml = (double*)malloc(sizeof(double) * N);
    double* up_bin = (double*)calloc((size_t)L * (n + 1), sizeof(double));
    double* dn_bin = (double*)calloc((size_t)L * (n + 1), sizeof(double));
    int bad = 0;

    ref_grid(a, lp, Pp, dm, NULL);
    ref_gauss_legendre(G, gx, gw);
    ref_boundary_spectra(a, toa, bint);
    /* opacity sample points: the column's points (sublayered grid) or the layer
     * centres (isothermal grid) */
    const int nq = iso ? n : np;
    if (iso) {
        for (int i = 0; i < n; ++i) {
            Tq[i] = T[i];
            dml[i] = (Pp[2 * i] - Pp[2 * i + 2]) / a->grav;
            ref_table_coord(lp[2 * i + 1], a->log10P0, a->dlog10P, a->nP, &iP[i], &wP[i]);
        }
    } else {
        ref_point_temperatures(n, T, Tq);
        for (int q = 0; q < np; ++q) ref_table_coord(lp[q], a->log10P0, a->dlog10P, a->nP, &iP[q], &wP[q]);
    }
    for (int q = 0; q < nq; ++q) ref_table_coord(Tq[q], a->T0, a->dT, a->nT, &iT[q], &wT[q]);

#pragma omp parallel for schedule(dynamic, 2) reduction(| : bad)
    for (int l = 0; l < L; ++l) {
        const int M2 = 2 * N;
        double* B = (double*)malloc(sizeof(double) * nq);
        double* kap = (double*)malloc(sizeof(double) * nq);
        double* A = (double*)malloc(sizeof(double) * (size_t)M2 * M2);
        double* x = (double*)malloc(sizeof(double) * M2);
        const double g0 = a->g0[l];
        const double kR = a->rayleigh ? ref_rayleigh_kappa(a->nu_edges[l], a->nu_edges[l + 1], p->mbar_mp) : 0.0;
        for (int q = 0; q < nq; ++q) B[q] = bin_planck(a, l, Tq[q]);
        if (Fup_toa) Fup_toa[l] = 0.0;
        for (int g = 0; g < G; ++g) {
            const double wg = 0.5 * gw[g];
            for (int q = 0; q < nq; ++q) {
                int i1 = a->nP > 1 ? iP[q] + 1 : iP[q], j1 = a->nT > 1 ? iT[q] + 1 : iT[q];
                double k00 = table_value(a, iP[q], iT[q], l, g), k10 = table_value(a, i1, iT[q], l, g);
                double k01 = table_value(a, iP[q], j1, l, g), k11 = table_value(a, i1, j1, l, g);
                kap[q] = (1.0 - wT[q]) * ((1.0 - wP[q]) * k00 + wP[q] * k10)
                       + wT[q] * ((1.0 - wP[q]) * k01 + wP[q] * k11);
            }
            memset(A, 0, sizeof(double) * (size_t)M2 * M2);
            A[0] = 1.0; A[1] = -1.0; x[0] = bint[l];                    /* eq. (22) */
            for (int s = 0; s < N - 1; ++s) {
                double c[6];
                const double kabs = iso ? kap[s] : 0.5 * (kap[s] + kap[s + 1]);
                const double w0 = a->rayleigh ? kR / (kabs + kR) : a->omega0[l];       /* Sect. 2.1.4 */
                if (iso) iso_affine(B[s], (kabs + kR) * dml[s], w0, g0, p, c);
                else ref_layer_affine(B[s], B[s + 1], (kabs + kR) * dm[s], w0, g0, p, c);
                double* ru = A + (size_t)(2 * s + 1) * M2;              /* F_up,s+1 equation */
                ru[2 * s + 2] = 1.0; ru[2 * s] = -c[0]; ru[2 * s + 3] = -c[1]; x[2 * s + 1] = c[2];
                double* rd = A + (size_t)(2 * s + 2) * M2;              /* F_dn,s equation */
                rd[2 * s + 1] = 1.0; rd[2 * s + 3] = -c[3]; rd[2 * s] = -c[4]; x[2 * s + 2] = c[5];
            }
            A[(size_t)(M2 - 1) * M2 + (M2 - 1)] = 1.0; x[M2 - 1] = toa[l];    /* eq. (20) */
            if (band_solve(M2, 2, 2, A, x) != 0) { bad = 1; continue; }
            /* interface fluxes: every point of the isothermal grid, the even points
             * of the sublayered grid */
            for (int i = 0; i <= n; ++i) {
                const int k = iso ? i : 2 * i;
                up_bin[(size_t)l * (n + 1) + i] += wg * x[2 * k];
                dn_bin[(size_t)l * (n + 1) + i] += wg * x[2 * k + 1];
                if (!isfinite(x[2 * k]) || !isfinite(x[2 * k + 1])) bad = 1;
            }
            if (Fup_toa) Fup_toa[l] += wg * x[2 * (N - 1)];
        }
        free(B); free(kap); free(A); free(x);
    }
    for (int i = 0; i <= n; ++i) {
        double su = 0.0, sd = 0.0;
        for (int l = 0; l < L; ++l) {
            su += up_bin[(size_t)l * (n + 1) + i];
            sd += dn_bin[(size_t)l * (n + 1) + i];
        }
        Fup_bol[i] = su;
        Fdn_bol[i] = sd;
    }
    free(lp); free(Pp); free(dm); free(Tq); free(gx); free(gw); free(toa); free(bint);
    free(iP); free(iT); free(wP); free(wT); free(dml); free(up_bin); free(dn_bin);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* One radiative-equilibrium temperature step, Sects. 2.2.3-2.2.4.
 *
 * Net flux F_- = F_up - F_dn at each interface; divergence of layer i
 * dF_i = F_-(i+1) - F_-(i) (eq. 23).  Convergence (eq. 29): every layer has
 * |dF_i| / (sigma T_i^4) < tol; then T is left unchanged and REF_CONVERGED is
 * returned.  Otherwise each layer takes the step of eq. (24) with
 *   rho_i = P_i mbar / (k_B T_i),  dz_i = k_B T_i/(mbar g) ln(P_int,i/P_int,i+1) (eq. 18),
 *   c_p = (2 + n_dof)/(2 mbar) k_B (eq. 25),
 *   dt_i = m_i f_pre t_rad (eq. 26), t_rad = c_p P_i/(sigma g T_i^3) (eq. 27),
 *   f_pre = 1e5 / |dF_i|^0.9 (eq. 28),
 * and m_i the per-layer timestep multiplier of the oscillation control.
 * Reading of the sign of eq. (24): dT_i = -dt_i/(rho_i c_p) * dF_i/dz_i, a
 * layer that loses more net flux through its top than it receives at its
 * bottom cools (the printed sign makes the iteration run away).
 * Oscillation control (Sect. 2.2.4; reading): the signs of the last 6
 * temperature changes are kept; once 6 are recorded, six equal signs (a
 * monotonic change) increase m_i by 10% (x1.1, capped at mult_max) and any
 * sign change among them counts as an oscillation and reduces m_i by 33%
 * (x0.67).  The paper makes the two cases complementary ("no oscillations
 * ... i.e. monotonic"); treating only strict alternation as an oscillation
 * leaves period-4 cycles (++--) undamped forever.  T is floored at T_floor.
 * hist bit 0 is the newest sign (1 = positive change). */
int ref_temp_update(const ref_atm* a, const ref_params* p, const double* Fup_bol, const double* Fdn_bol,
                    double* T, double* mult, int* hist, int* nhist, double* metric, double* dT)
{
    const int n = a->n;
    double* P = (double*)malloc(sizeof(double) * (2 * n + 1));
    ref_grid(a, NULL, P, NULL, NULL);
    const double mbar = p->mbar_mp * M_PROTON;
    const double cp = (2.0 + p->n_dof) / (2.0 * mbar) * K_B;
    double worst = 0.0;
    int nonfinite = 0;
    for (int i = 0; i < n; ++i) {
        double dF = (Fup_bol[i + 1] - Fdn_bol[i + 1]) - (Fup_bol[i] - Fdn_bol[i]);
        double m = fabs(dF) / (SIGMA_SB * pow(T[i], 4));
        if (!isfinite(m)) nonfinite = 1;
        if (m > worst) worst = m;
    }
    if (metric) *metric = worst;
    if (nonfinite) { free(P); return REF_NONFINITE; }
    if (worst < p->tol) {
        if (dT) for (int i = 0; i < n; ++i) dT[i] = 0.0;
        free(P);
        return REF_CONVERGED;
    }
    for (int i = 0; i < n; ++i) {
        double dF = (Fup_bol[i + 1] - Fdn_bol[i + 1]) - (Fup_bol[i] - Fdn_bol[i]);
        double Pi = P[2 * i + 1];
        double rho = Pi * mbar / (K_B * T[i]);
        double dz = K_B * T[i] / (mbar * a->grav) * log(P[2 * i] / P[2 * i + 2]);
        double trad = cp * Pi / (SIGMA_SB * a->grav * pow(T[i], 3));
        double step = 0.0;
        if (dF != 0.0) {
            double fpre = p->fpre_num / pow(fabs(dF), p->fpre_exp);
            double dt = mult[i] * fpre * trad;
            step = -(1.0 / (rho * cp)) * (dF / dz) * dt;
        }
        double Tn = T[i] + step;
        if (Tn < p->T_floor) Tn = p->T_floor;
        if (dT) dT[i] = Tn - T[i];
        T[i] = Tn;
        hist[i] = ((hist[i] << 1) | (step > 0.0 ? 1 : 0)) & 0x3F;
        if (nhist[i] < 6) nhist[i] += 1;
        if (nhist[i] >= 6) {
            if (hist[i] == 0x00 || hist[i] == 0x3F) {
                mult[i] *= p->osc_up;
                if (mult[i] > p->mult_max) mult[i] = p->mult_max;
            } else {
                mult[i] *= p->osc_down;
            }
        }
    }
    free(P);
    /* with the tables of Sect. 2.6, a temperature above the Planck table's last node would take
       that node's values: the iteration stops instead */
    if (p->tabulate)
        for (int i = 0; i < n; ++i)
            if (!(T[i] <= REF_TAB_DT * (REF_TAB_NT - 1))) return REF_OUT_OF_RANGE;
    return REF_UPDATED;
}

/* The radiative-equilibrium iteration of Sect. 2.2.3: alternate a full flux
 * evaluation and a temperature step until eq. (29) holds in every layer or
 * max_iter flux evaluations have been made.  mult/hist/nhist/warm carry the
 * iteration state (NULL: fresh state owned here; a zeroed warm buffer is the
 * same as a cold start).  iters = number of flux evaluations. */
int ref_solve_re(const ref_atm* a, const ref_params* p, double* T, double* mult, int* hist, int* nhist,
                 double* warm, int* iters, double* metric)
{
    const int n = a->n, np = 2 * n + 1;
    const int K = ref_passes(a, p);
    double* m_own = NULL;
    int* h_own = NULL;
    int* c_own = NULL;
    double* w_own = NULL;
    if (!mult) { mult = m_own = (double*)malloc(sizeof(double) * n); for (int i = 0; i < n; ++i) mult[i] = 1.0; }
    if (!hist) { hist = h_own = (int*)calloc(n, sizeof(int)); }
    if (!nhist) { nhist = c_own = (int*)calloc(n, sizeof(int)); }
    if (!warm) { warm = w_own = (double*)calloc((size_t)a->L * a->G * np, sizeof(double)); }
    double* Fu = (double*)malloc(sizeof(double) * (n + 1));
    double* Fd = (double*)malloc(sizeof(double) * (n + 1));
    int status = REF_NOT_CONVERGED, it;
    for (it = 0; it < p->max_iter; ++it) {
        if (ref_flux_sweep(a, p, T, K, 0, warm, 1, Fu, Fd, NULL, NULL, NULL) != 0) {
            status = REF_NONFINITE;
            ++it;
            break;
        }
        int st = ref_temp_update(a, p, Fu, Fd, T, mult, hist, nhist, metric, NULL);
        if (st == REF_CONVERGED) { status = REF_CONVERGED; ++it; break; }
        if (st == REF_NONFINITE) { status = REF_NONFINITE; ++it; break; }
        if (st == REF_OUT_OF_RANGE) { status = REF_OUT_OF_RANGE; ++it; break; }
    }
    if (iters) *iters = it;
    free(Fu); free(Fd); free(m_own); free(h_own); free(c_own); free(w_own);
    return status;
}
