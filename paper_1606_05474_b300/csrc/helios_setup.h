// Host-side set-up shared by helios_plan_create (helios_api.cu) and helios_flux_sweep_noalloc
// (helios_noalloc.cu): constants, the pressure grid of an atmosphere, the Gauss-Legendre weights
// and the per-bin constants, all in double precision and then rounded.
//
// Include after <cmath>, <cstring>, helios.h and helios_kernels.cuh, in the namespace that holds
// that copy of the device structs (BinConst); this header includes nothing itself.

namespace helios_setup {

// CODATA 2018, CGS
constexpr double kB = 1.380649e-16;
constexpr double hP = 6.62607015e-27;
constexpr double cL = 2.99792458e10;
constexpr double sigmaSB = 5.670374419e-5;
constexpr double kPi = 3.14159265358979323846;
constexpr double mProton = 1.67262192369e-24;
constexpr double mbarMp = 2.4;        // mean molecular mass in proton masses (Sect. 2.2.1)

// IEEE double table coordinate, the same formula as the device code (no contraction: the files
// including this are compiled with -ffp-contract=off for the host)
inline void host_table_coord(double x, double x0, double dx, int nx, int& i, double& w)
{
    if (nx < 2) { i = 0; w = 0.0; return; }
    const double u = (x - x0) / dx;
    if (!(u > 0.0)) i = 0;
    else if (u >= (double)(nx - 2)) i = nx - 2;
    else i = (int)std::floor(u);
    double t = (x - (x0 + (double)i * dx)) / dx;
    if (!(t > 0.0)) t = 0.0;
    if (t > 1.0) t = 1.0;
    w = t;
}

// Gauss-Legendre weights on [0, 1] (eqs. 31-32, with the 1/2 of eq. 31): nodes of P_G by Newton
// iteration in long double from Tricomi's initial approximation, w = 1 / ((1 - y^2) P_G'(y)^2),
// ascending nodes
inline void gauss_weights01(int G, float* w01)
{
    if (G == 1) { w01[0] = 1.0f; return; }
    for (int k = 1; k <= G; ++k) {
        const long double th = kPi * (4.0L * k - 1.0L) / (4.0L * G + 2.0L);
        long double x = (1.0L - (G - 1.0L) / (8.0L * G * G * G)) * cosl(th);
        long double dP = 1.0L;
        for (int it = 0; it < 60; ++it) {
            long double pm = 1.0L, pc = x;
            for (int j = 2; j <= G; ++j) {
                const long double pn = ((2.0L * j - 1.0L) * x * pc - (j - 1.0L) * pm) / j;
                pm = pc;
                pc = pn;
            }
            dP = G * (pm - x * pc) / (1.0L - x * x);
            const long double dx = pc / dP;
            x -= dx;
            if (fabsl(dx) < 1e-19L) break;
        }
        w01[G - k] = (float)(0.5 * (double)(2.0L / ((1.0L - x * x) * dP * dP)));
    }
}

// Planck intensity of a wavenumber bin at its centre, times the bin width (per steradian)
inline double planck_bin(double nu_lo, double nu_hi, double T)
{
    if (!(T > 0.0)) return 0.0;
    const double nu = 0.5 * (nu_lo + nu_hi), dnu = nu_hi - nu_lo;
    return 2.0 * hP * cL * cL * nu * nu * nu * dnu / std::expm1(hP * cL * nu / (kB * T));
}

// Pressure grid of an n-layer atmosphere (Sect. 2.2.1, eq. 19): layer centres log-spaced from
// P_bot to P_top, interfaces at the geometric means, the outer ones half a step beyond; per point
// the pressure-table coordinate, per sublayer the column mass, per layer ln(P_i / P_i+1).
// iso_layers: both points of layer i sit at its centre pressure, sublayer 2i is the whole layer
// and sublayer 2i+1 a zero-thickness step.  P: scratch of 2n+1 doubles.
inline void layer_geometry(int n, double P_bot_bar, double P_top_bar, double grav, int iso_layers,
                           const helios_ktable_t& k, double* P, int* iP, double* wP, float* dm, double* lnr)
{
    const double lb = std::log10(P_bot_bar), lt = std::log10(P_top_bar);
    const double h = (lb - lt) / (double)(n - 1);
    for (int p = 0; p <= 2 * n; ++p) {
        const double lp = (lb + 0.5 * h) - (0.5 * h) * (double)p;
        P[p] = 1e6 * std::pow(10.0, lp);
        const double lq = iso_layers ? lb - h * (double)(p >> 1 < n - 1 ? p >> 1 : n - 1) : lp;
        host_table_coord(lq, k.log10P0, k.dlog10P, k.nP, iP[p], wP[p]);
    }
    for (int s = 0; s < 2 * n; ++s) {
        const double dP = iso_layers ? ((s & 1) ? 0.0 : P[s] - P[s + 2]) : P[s] - P[s + 1];
        dm[s] = (float)(dP / grav);
    }
    for (int i = 0; i < n; ++i) lnr[i] = std::log(P[2 * i] / P[2 * i + 2]);
}

// Per-bin constants of one atmosphere's L bins (eqs. 8, 12-14, 20-22; Sect. 2.1.4 for Rayleigh
// scattering): Planck prefactors, the incident and internal fluxes spread over the bins like
// blackbodies at T_star and T_int (normalised to sigma T_irr^4 and sigma T_int^4), and the
// two-stream constants.  e: L + 1 edges (cm^-1).  Returns whether any bin scatters.
inline bool bin_constants(const double* e, const float* omega0, const float* g0s, int L, double T_irr, double T_int,
                          double T_star, const helios_params_t& prm, helios_dev::BinConst* out)
{
    using namespace helios_dev;
    const double D = prm.D, eps = 1.0 / D;
    double s_star = 0.0, s_int = 0.0;
    for (int l = 0; l < L; ++l) {
        s_star += planck_bin(e[l], e[l + 1], T_star);
        s_int += planck_bin(e[l], e[l + 1], T_int);
    }
    const double Firr = sigmaSB * std::pow(T_irr, 4), Fint = sigmaSB * std::pow(T_int, 4);
    bool any_scat = false;
    for (int l = 0; l < L; ++l) {
        BinConst& c = out[l];
        std::memset(&c, 0, sizeof c);
        const double nu = 0.5 * (e[l] + e[l + 1]), dnu = e[l + 1] - e[l];
        const double xs = hP * cL * nu / kB;
        c.xs = (float)xs;
        c.xs_lo = (float)(xs - (double)c.xs);
        c.E = (float)(2.0 * kPi * eps * 2.0 * hP * cL * cL * nu * nu * nu * dnu);
        double toa = (s_star > 0.0 && Firr > 0.0) ? Firr * planck_bin(e[l], e[l + 1], T_star) / s_star : 0.0;
        double bint = (s_int > 0.0 && Fint > 0.0) ? Fint * planck_bin(e[l], e[l + 1], T_int) / s_int : 0.0;
        if (prm.grey_mode) {
            if (l == 0) { c.flags |= BIN_GREY_DARK; toa = Firr; bint = 0.0; }
            else { c.flags |= BIN_GREY_THERM; c.E = (float)(eps * sigmaSB); toa = 0.0; bint = Fint; }
        }
        c.toa = (float)toa;
        c.bint = (float)bint;
        const double g0 = g0s[l];
        if (prm.rayleigh) {
            // Sect. 2.1.4, eqs. (16)-(17): H2 cross section at the bin centre over mbar; the
            // sublayer constants follow from it in the sweep (rayleigh_const)
            const double lam_cm = 1.0 / nu;
            const double nr = 13.58e-5 * (1.0 + 7.52e-11 / (lam_cm * lam_cm)) + 1.0;
            const double f = (nr * nr - 1.0) / (nr * nr + 2.0), nref = 2.68678e19;
            const double sig = 24.0 * kPi * kPi * kPi / (nref * nref * lam_cm * lam_cm * lam_cm * lam_cm) * f * f;
            c.flags |= BIN_RAYLEIGH;
            c.lam = (float)(sig / (mbarMp * mProton));
            c.q = (float)g0;
            c.gam = (float)(D * (1.0 - g0) / 2.0);
            any_scat = true;
            continue;
        }
        const double w0 = omega0[l];
        if (w0 != 0.0) any_scat = true;
        if (1.0 - w0 < prm.w0_pure) c.flags |= BIN_PURE_SCAT;
        if (w0 == 0.0) c.flags |= BIN_NO_SCAT;
        const double one_wg = 1.0 - w0 * g0;
        const double lam = D * std::sqrt(one_wg * (1.0 - w0));
        c.lam = (float)lam;
        const double kk = one_wg > 0.0 ? std::sqrt((1.0 - w0) / one_wg) : 0.0;
        const double q = (1.0 - kk) / (1.0 + kk);
        const double omq = 2.0 * kk / (1.0 + kk), omq2 = omq * (1.0 + q);     // 1 - q, 1 - q^2
        // S = eps/(1 - w0 g0) dB (1 - Ts + Rs)/dtau and (1 - Ts + Rs)/dtau = lam phi h
        const double cl = lam * eps / (prm.printed_gradient ? (1.0 + w0 * g0) : one_wg);
        c.q = (float)q;
        c.cl = (float)cl;
        if (kk > 0.0) {                     // (kk = 0: conservative scattering, the eq. 14 branch)
            c.c2 = (float)(q * q / omq2);
            c.qo = (float)(q / omq2);
            c.hoh = (float)(0.5 / omq);
            c.clh = (float)(cl / omq);
        }
        c.gam = (float)(D * (1.0 - g0) / 2.0);
    }
    return any_scat;
}

}  // namespace helios_setup
