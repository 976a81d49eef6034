// Device kernels of the radiative-equilibrium hot path (sm_103a).
//
// One flux evaluation + temperature step (helios_flux_sweep + helios_temp_update) is four
// launches; helios_re_step fuses finalize and temp into post_kernel (three), and inside
// helios_solve_re post_kernel also does the next step's prep (two: sweep + post):
//   prep_kernel      one thread per point: point temperatures (Sect. 2.2.1),
//                    temperature-table coordinates in IEEE double (Sect. 2.3), the
//                    table row offset and the four bilinear weights of the point, and
//                    the float inputs of the Planck evaluations.
//   sweep_kernel<M>  one block per work item = (atmosphere, tile of bins); one warp
//                    per Gauss point g, so a block holds the G columns of one bin at a
//                    time.  The 2n sublayers of a column are spread over the 32 lanes of
//                    its warp (M consecutive sublayers per lane); their two-stream
//                    coefficients stay in registers for all passes, and each down or up
//                    sweep is a first-order linear recurrence solved as a warp-wide affine
//                    scan (lane-local composition, 5 shuffle levels, lane-local apply).
//   finalize_kernel  one warp per interface: fixed-order FP64 sums of the per-item
//                    partials -> bolometric fluxes (deterministic).
//   temp_kernel      one block per atmosphere, a thread per layer: net-flux divergence,
//                    the convergence metric of eq. (29) reduced with an exact max, the
//                    convergence decision and the FP64 temperature step of eqs. (24)-(28)
//                    with the oscillation rule.
//   post_kernel      one block per atmosphere: finalize + temp (+ prep of the next step).
//
// Fluxes are carried in the sweep as deviations from the local two-stream Planck flux,
// G = F - 2 pi eps B_l(T_p).  With per-sublayer transmission Ts, reflection Rs and
// source Ss the layer solutions of eqs. (11), (14) and (15) become
//     G_top,up   = Ts G_bot,up + Rs G_top,dn + Ss
//     G_bot,dn   = Ts G_top,dn + Rs G_bot,up - Ss
// (an exact algebraic rewrite), so the net flux G_up - G_dn = F_up - F_dn never forms
// the difference of two large float numbers, and every source term is a product of the
// small Planck difference across the sublayer, evaluated from the temperature
// difference (formed in double precision) without cancellation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace helios_dev {

constexpr unsigned FULL = 0xffffffffu;

// per-bin flags
constexpr int BIN_PURE_SCAT = 1;    // 1 - omega0 < w0_pure: eq. (14), no thermal source
constexpr int BIN_NO_SCAT = 2;      // omega0 == 0: streams decouple, one pass is exact
constexpr int BIN_GREY_DARK = 4;    // grey mode visible band: no emission
constexpr int BIN_GREY_THERM = 8;   // grey mode thermal band: pi B = sigma T^4
constexpr int BIN_RAYLEIGH = 16;    // H2 Rayleigh opacity kappa_R (in `lam`) added to every sublayer;
                                    // omega0 per sublayer and g (g0 in `q`), constants per sublayer

struct __align__(16) BinConst {
    float xs;      // h c nu_c / k_B  (x = xs / T), high part
    float xs_lo;   // low part of h c nu_c / k_B (float-float)
    float E;       // 2 pi eps * 2 h c^2 nu_c^3 dnu  (2 pi eps B_l(T) = E / (e^x - 1)); eps sigma in grey mode
    float toa;     // downward flux entering at the TOA (eq. 20)
    float bint;    // internal flux entering at the BOA (eq. 22)
    float lam;     // D sqrt((1 - w0 g0)(1 - w0))  (eq. 8 exponent per unit dtau)
    float q;       // zeta_- / zeta_+  (eq. 13)
    float c2;      // q^2 / (1 - q^2)
    float qo;      // q / (1 - q^2)
    float hoh;     // 1 / (2 (1 - q))
    float cl;      // lam * eps / (1 - w0 g0): gradient prefactor of eq. (15) times lam
    float clh;     // cl / (1 - q)
    float gam;     // D (1 - g0) / 2: pure-scattering coupling, eq. (14)
    int flags;
    float pad[2];
};

struct AtmDesc {
    int n, L, M, tab;       // M: lane chunk of the iterated sweep's layout (cl lanes per column)
    int lay_off, if_off, pt_off, sub_off;
    int bin_off, item_off, n_items, n_spec;   // n_spec > 1: opacity mixed from several tables
    int spec_off, cl, pad1, pad2;             // cl: lanes per column of the iterated sweep (16, 32)
    long long warm_off;     // float offset of this atmosphere's warm-start block
    long long part_off;     // double offset of this atmosphere's partial sums
    long long fspec_off;    // float offset of this atmosphere's per-bin flux block [L][2][2n+1]
};

struct TabDesc {
    const float* kappa;
    int nP, nT, L, G;
    double log10P0, dlog10P, T0, dT;
    int rowL;               // L * G: floats per (iP, iT) row
    int offP;               // offset to the next pressure node (0 if nP == 1)
    int offT;               // offset to the next temperature node (0 if nT == 1)
    int pad;
};

struct PlanDev {
    const AtmDesc* atms;
    const TabDesc* tabs;
    const BinConst* bins;
    const int2* items;          // (atm, tile)
    const float* gw;            // Gauss weights on [0, 1], [G]
    const int* iP;              // [points]
    const double* wP;           // [points]
    const float* dm;            // [sublayers]  column mass (g cm^-2)
    const double* lnr;          // [layers]  ln(P_int,i / P_int,i+1)
    const int* lay_atm;         // [layers] atmosphere of each layer
    const int* spec_tab;        // species tables of mixed-opacity atmospheres (eq. 34)
    const float* spec_w;        // their mass mixing ratios (eq. 35)
    // per-evaluation state written by prep_kernel
    double* Tpt;                // [points] temperature at the point in the previous evaluation
    int* iT;                    // [points]
    double* wT;                 // [points]
    int* row;                   // [points] table offset of corner (iP, iT) for bin 0, g 0
    float4* wq;                 // [points] bilinear weights (00, P+1, T+1, both)
    float2* invT;               // [points] 1/T as a float-float pair
    float* Tf;                  // [points] T (grey mode)
    float2* invT_old;           // [points] 1/T of the previous evaluation, float-float
    float* dinv_step;           // [points] (T_old - T)/(T_old T)
    float* dT_step;             // [points] T_old - T (grey mode)
    float* dinv_sub;            // [sublayers] (T_a - T_b)/(T_a T_b), a below b
    float* dT_sub;              // [sublayers] T_a - T_b (grey mode)
    float* warm;                // warm-start G_up per column, lane-interleaved
    double* part;               // per-item partial sums [3][n+1]
    int G, TB, A;
    float dtau_iso;             // at least FLT_MIN: a zero-thickness sublayer takes the isothermal form
    float D, eps, w0_pure;      // per-sublayer two-stream constants (Rayleigh scattering)
    int printed_gradient;
    int iso_layers;             // 1: isothermal-layer grid (both points of layer i at T_i)
    // tables of Sect. 2.6 (null: the functions themselves): 1 - e^-x at the nodes
    // x_i = 10^(kTabX0 + 0.1 i) ([0, kTabNX): x_i, [kTabNX, 2 kTabNX): 1 - e^-x_i), and each bin's
    // 2 pi eps B_l at the nodes T_j = j kTabDT ([bins][kTabNT])
    const float* utab;
    const float* btab;
};

constexpr float kTabX0 = -8.05f;
constexpr int kTabNX = 102;
constexpr float kTabDT = 10.0f;
constexpr int kTabNT = 601;

// ---------------------------------------------------------------------------
// Table coordinate in IEEE double without contraction (Sect. 2.3 and footnote):
// i = clamp(floor((x - x0)/dx), 0, nx-2), w = clamp((x - (x0 + i dx))/dx, 0, 1).
__device__ __forceinline__ void table_coord(double x, double x0, double dx, int nx, int& i, double& w)
{
    if (nx < 2) { i = 0; w = 0.0; return; }
    double u = __ddiv_rn(__dsub_rn(x, x0), dx);
    if (!(u > 0.0)) i = 0;
    else if (u >= (double)(nx - 2)) i = nx - 2;
    else i = (int)floor(u);
    double t = __ddiv_rn(__dsub_rn(x, __dadd_rn(x0, __dmul_rn((double)i, dx))), dx);
    if (!(t > 0.0)) t = 0.0;
    if (t > 1.0) t = 1.0;
    w = t;
}

// temperature at point p of an n-layer column (Sect. 2.2.1; outer interfaces take the
// nearest centre)
__device__ __forceinline__ double point_T(const double* T, int n, int p, int iso_layers)
{
    // isothermal layers (Sect. 2.2.1): points 2i and 2i+1 bound layer i and carry its
    // temperature; the last point repeats the top layer
    if (iso_layers) return T[min(p >> 1, n - 1)];
    if (p & 1) return T[p >> 1];
    int i = p >> 1;
    if (i == 0) return T[0];
    if (i == n) return T[n - 1];
    return __dmul_rn(0.5, __dadd_rn(T[i - 1], T[i]));
}

// corner offset and the four bilinear weights of a point; all weights non-negative
// and formed in double, so no cancellation when corners differ by decades
__device__ __forceinline__ void point_corners(const TabDesc& td, int iP, double wP, int iT, double wT, int& row,
                                              float4& wq)
{
    row = (iP * td.nT + iT) * td.rowL;
    const double p1 = wP, p0 = 1.0 - wP, t1 = wT, t0 = 1.0 - wT;
    wq = make_float4((float)(t0 * p0), (float)(t0 * p1), (float)(t1 * p0), (float)(t1 * p1));
}

__device__ __forceinline__ float kappa_at(const float* __restrict__ tab, const TabDesc& td, int row, float4 w, int lg)
{
    const float* r = tab + row + lg;
    const float k00 = __ldg(r), k10 = __ldg(r + td.offP), k01 = __ldg(r + td.offT), k11 = __ldg(r + td.offP + td.offT);
    return fmaf(w.w, k11, fmaf(w.z, k01, fmaf(w.y, k10, w.x * k00)));
}

// e^x - 1 with full relative accuracy: Taylor series to x^9 for |x| < 0.35 (truncation
// below 3e-10), otherwise expf(x) - 1 (no cancellation there: |e^x - 1| > 0.29).
__device__ __forceinline__ float em1(float x)
{
    if (fabsf(x) < 0.35f) {
        float p = fmaf(x, 2.7557319e-6f, 2.4801587e-5f);
        p = fmaf(x, p, 1.9841270e-4f);
        p = fmaf(x, p, 1.3888889e-3f);
        p = fmaf(x, p, 8.3333333e-3f);
        p = fmaf(x, p, 4.1666667e-2f);
        p = fmaf(x, p, 1.6666667e-1f);
        p = fmaf(x, p, 0.5f);
        p = fmaf(x, p, 1.0f);
        return x * p;
    }
    return expf(x) - 1.0f;
}

// phi(x) = (1 - e^{-x})/x for x >= 0 (Taylor series below 0.35, else direct), with
// u = 1 - e^{-x} = x phi and t = e^{-x}.  Both forms are evaluated and selected: a lane's
// sublayers lie at every depth of the column, so a branch would split every warp.  phi enters
// only the source term, where a rounding bias does not compound along the column, so the
// quotient may use the approximate divide
__device__ __forceinline__ void phi_u_t(float x, float& phi, float& u, float& t)
{
    float p = fmaf(x, -2.4801587e-5f, 1.9841270e-4f);         // (-1)^k x^k / (k+1)!
    p = fmaf(x, p, -1.3888889e-3f);
    p = fmaf(x, p, 8.3333333e-3f);
    p = fmaf(x, p, -4.1666667e-2f);
    p = fmaf(x, p, 1.6666667e-1f);
    p = fmaf(x, p, -0.5f);
    const float ph = fmaf(x, p, 1.0f);
    const float te = expf(-x);             // accurate to ~1 ulp for any x (the fast intrinsic's
    const float ue = 1.0f - te;            // error grows with |x| and compounds through transmissions)
    const bool small = x < 0.35f;
    u = small ? x * ph : ue;
    t = small ? 1.0f - u : te;
    phi = small ? ph : __fdividef(ue, x);
}

// 1/a for a normal positive a: the hardware's approximate reciprocal refined by one
// Newton-Raphson step in FMA form, r' = r + r (1 - a r) (Markstein, IBM J. Res. Dev. 34, 1990).
// Within one unit in the last place of the correctly rounded quotient and without a bias in
// the direction of its errors (both checked against correctly rounded quotients), in three
// instructions and no branch
__device__ __forceinline__ float recip_nr(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return fmaf(r, fmaf(-a, r, 1.0f), r);
}

__global__ void recip_kernel(const float* __restrict__ x, float* __restrict__ y, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = recip_nr(x[i]);
}

// phi, u = 1 - e^{-x} and t = e^{-x} with u from the table of Sect. 2.6: linear in x between the
// 0.1-dex nodes, x itself below the first node, 1 above the last; phi = u / x
__device__ __forceinline__ void phi_u_t_tab(float x, const float* __restrict__ utab, float& phi, float& u, float& t)
{
    const float f = (__log10f(fmaxf(x, 1e-30f)) - kTabX0) * 10.0f;
    const int i = (int)floorf(f);
    if (i < 0) {
        u = x;
    } else if (i >= kTabNX - 1) {
        u = 1.0f;
    } else {
        const float x0 = __ldg(utab + i), x1 = __ldg(utab + i + 1);
        const float u0 = __ldg(utab + kTabNX + i), u1 = __ldg(utab + kTabNX + i + 1);
        u = fmaf(__fdividef(x - x0, x1 - x0), u1 - u0, u0);
    }
    t = 1.0f - u;
    phi = x > 0.0f ? __fdividef(u, x) : 1.0f;
}

// 2 pi eps B of a bin at temperature T from its 10 K table (linear in T, end nodes beyond)
__device__ __forceinline__ float planck_tab(const float* __restrict__ row, float T)
{
    const float f = T * (1.0f / kTabDT);
    const int j = min(max((int)floorf(f), 0), kTabNT - 2);
    const float w = fminf(fmaxf(f - (float)j, 0.0f), 1.0f);
    const float b0 = __ldg(row + j), b1 = __ldg(row + j + 1);
    return fmaf(w, b1 - b0, b0);
}

// a + b for float-float values (hi, lo): Knuth's error-free two-sum of the high parts plus the
// low parts, renormalised
__device__ __forceinline__ float2 ff_add(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float v = s - a.x;
    const float e = ((a.x - (s - v)) + (b.x - v)) + (a.y + b.y);
    const float h = s + e;
    return make_float2(h, e - (h - s));
}

// Two-stream Planck flux E / (e^x - 1) of a bin at 1/T = it (float-float), with x = xs / T
// formed as an error-free float-float product so that the Wien tail keeps full relative
// accuracy (B ~ e^{-x} amplifies an error in x by x).  Returns the high part of x in xh.
__device__ __forceinline__ float planck_ff(const BinConst& b, float2 it, float& xh)
{
    const float p = b.xs * it.x;
    const float lo = fmaf(b.xs, it.y, fmaf(b.xs_lo, it.x, fmaf(b.xs, it.x, -p)));
    xh = p;
    if (p > 80.0f) return 0.0f;                       // below 1e-34 E
    float em;
    if (p < 0.35f) {
        em = em1(p + lo);
    } else {
        const float ex = expf(p);
        em = fmaf(ex, lo, ex - 1.0f);                 // e^{p + lo} - 1, |lo| ~ 1e-7 p
    }
    return __fdividef(b.E, em);
}

// a hint to bring the line holding p into L2 (generic address; no effect on results)
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.L2 [%0];" ::"l"(p));
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of one evaluation (prep, sweep, finalize, post)
// may be launched to start while their predecessor in the stream is still running: each one
// first lets its own successor launch, then waits until its predecessor has completed and its
// memory is visible, before it reads or writes anything.  Launched the ordinary way, both are
// no-ops.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// point quantities of point p of atmosphere ad at the temperatures T_layer (warm_valid: the
// previous evaluation's point temperature is the old one of the warm-start shift)
__device__ __forceinline__ void prep_point(const PlanDev& P, const double* __restrict__ T_layer, const AtmDesc& ad,
                                           int p, int warm_valid)
{
    const int n = ad.n;
    const TabDesc td = P.tabs[ad.tab];
    const double* T = T_layer + ad.lay_off;
    const int q = ad.pt_off + p;
    const double Tn = point_T(T, n, p, P.iso_layers);
    int it, row;
    double w;
    float4 wq;
    table_coord(Tn, td.T0, td.dT, td.nT, it, w);
    point_corners(td, P.iP[q], P.wP[q], it, w, row, wq);
    P.iT[q] = it;
    P.wT[q] = w;
    P.row[q] = row;
    P.wq[q] = wq;
    const double To = warm_valid ? P.Tpt[q] : Tn;
    const float Tnf = (float)Tn, Tof = (float)To;
    const double in = 1.0 / Tn, io = 1.0 / To;
    const float inh = (float)in, ioh = (float)io;
    P.invT[q] = make_float2(inh, (float)(in - (double)inh));
    P.Tf[q] = Tnf;
    P.invT_old[q] = make_float2(ioh, (float)(io - (double)ioh));
    P.dinv_step[q] = (float)(To - Tn) / (Tof * Tnf);
    P.dT_step[q] = (float)(To - Tn);
    P.Tpt[q] = Tn;
    if (p < 2 * n) {
        const double Tb = point_T(T, n, p + 1, P.iso_layers);
        const float Tbf = (float)Tb;
        P.dinv_sub[ad.sub_off + p] = (float)(Tn - Tb) / (Tnf * Tbf);
        P.dT_sub[ad.sub_off + p] = (float)(Tn - Tb);
    }
}

__global__ void prep_kernel(PlanDev P, const double* __restrict__ T_layer, const int* __restrict__ status,
                            int warm_valid)
{
    pdl_enter();
    const int a = blockIdx.y;
    if (status && status[a] != 0) return;
    const AtmDesc ad = P.atms[a];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 2 * ad.n + 1) return;
    prep_point(P, T_layer, ad, p, warm_valid);
}

// Two-stream constants of one sublayer of a Rayleigh bin (Sect. 2.1.4): the H2 opacity kappa_R
// joins the sublayer's absorption opacity kabs, and omega0 = kappa_R / (kabs + kappa_R).
// 1 - omega0 = kabs/kt and 1 - omega0 g0 = (kabs + kappa_R (1 - g0))/kt are formed from the
// opacities (no cancellation), as is 1 - r = kappa_R (1 - g0)/(kt (1 - omega0 g0)(1 + r)), so
// q = zeta_-/zeta_+ = (1 - r)/(1 + r) keeps relative accuracy when scattering is weak.
// Returns the constants in a BinConst (flags: pure scattering or not) and the total opacity kt.
__device__ __forceinline__ BinConst rayleigh_const(const BinConst& b, const PlanDev& P, float kabs, float& kt)
{
    BinConst c = b;
    const float kR = b.lam, g0 = b.q;
    kt = kabs + kR;
    const float inv = __frcp_rn(kt);
    const float omw = kabs * inv;                               // 1 - omega0
    const float omwg = fmaf(kR, 1.0f - g0, kabs) * inv;         // 1 - omega0 g0
    c.flags = b.flags & ~BIN_RAYLEIGH;
    if (omw < P.w0_pure) {
        c.flags |= BIN_PURE_SCAT;
        return c;
    }
    const float r = sqrtf(__fdiv_rn(omw, omwg));
    const float omr = __fdiv_rn(kR * (1.0f - g0) * inv, omwg * (1.0f + r));
    const float q = __fdiv_rn(omr, 1.0f + r);
    c.lam = P.D * sqrtf(omwg * omw);                           // eq. (8)
    c.q = q;
    // with 1 - q = 2 r / (1 + r) and 1 - q^2 = 4 r / (1 + r)^2
    const float i4r = __frcp_rn(4.0f * r);
    c.hoh = (1.0f + r) * i4r;
    c.c2 = omr * omr * i4r;
    c.qo = omr * (1.0f + r) * i4r;
    c.cl = c.lam * __fdiv_rn(P.eps, P.printed_gradient ? fmaf(kR * inv, g0, 1.0f) : omwg);
    c.clh = 2.0f * c.cl * c.hoh;
    return c;
}

// Two-stream coefficients of one sublayer in deviation form (see file header).
// dB = 2 pi eps (B_bottom - B_top).
// With WANT_E the absorption Es = 1 - Ts - Rs of the sublayer is returned too, formed without
// cancellation: expanding eqs. (12)-(13), 1 - Ts - Rs = (1 - trans)(1 - q trans) d / (1 + q)
// (zero for pure scattering); eo = 1 / (1 + q) of the bin.
// A zero-thickness sublayer (the step between two isothermal layers, or a padding slot) gives
// exactly (1, 0, dB): trans = 1 and 1 - trans = 0 exactly, d = 1, and it takes the isothermal
// form (the threshold dtau_iso is at least the smallest normal float)
// KIND names the bin's kind when the caller knows it (its flags are uniform over a bin), so that
// the tests of the other kinds' branches drop out of an unrolled loop over the sublayers
enum { COEF_ANY = 0, COEF_GENERAL = 1, COEF_NO_SCAT = 2, COEF_PURE_SCAT = 3 };

template <bool WANT_E = false, bool TAB = false, int KIND = COEF_ANY>
__device__ __forceinline__ void layer_coef(const BinConst& b, float dtau, float dB, float dtau_iso,
                                           float& Ts, float& Rs, float& Ss, float* Es = nullptr, float eo = 0.0f,
                                           const float* utab = nullptr)
{
    if (KIND == COEF_PURE_SCAT || (KIND == COEF_ANY && (b.flags & BIN_PURE_SCAT))) {   // eq. (14): no thermal source
        const float a = b.gam * dtau;
        const float t = __frcp_rn(1.0f + a);
        Ts = t;
        Rs = a * t;
        // eq. (14) has no source, and Ts + Rs = 1: in deviation form G = F - 2 pi eps B the upward
        // stream gains Ts dB across the sublayer and the downward one loses it (zero in a
        // pure-scattering bin, where B = 0; not in a pure-scattering sublayer of a Rayleigh bin)
        Ss = t * dB;
        if constexpr (WANT_E) *Es = 0.0f;
        return;
    }
    float phi, u, tr;
    if constexpr (TAB) phi_u_t_tab(b.lam * dtau, utab, phi, u, tr);     // Sect. 2.6 table
    else phi_u_t(b.lam * dtau, phi, u, tr); // eq. (8): tr = exp(-lam dtau), u = 1 - tr
    const bool iso = dtau < dtau_iso;       // Sect. 2.2.1: thin sublayers use eq. (11)
    if (KIND == COEF_NO_SCAT || (KIND == COEF_ANY && (b.flags & BIN_NO_SCAT))) {   // zeta_- = 0: Ts = trans, Rs = 0
        Ts = tr;
        Rs = 0.0f;
        Ss = iso ? 0.5f * dB * (1.0f + tr) : b.cl * dB * phi;
        if constexpr (WANT_E) *Es = u;
        return;
    }
    // eqs. (12)-(13) divided by -zeta_+^2: Ts = xi/alpha, Rs = -beta/alpha, i.e. with
    // d = (1 - q^2) / (1 - q^2 trans^2) = 1 / (1 + c2 (1 - trans^2)):  Ts = trans d and
    // Rs = qo (1 - trans^2) d; the source term's (1 - Ts + Rs)/u = (1 + q - q u) d / (1 - q).
    // The reciprocal is accurate to an ulp without bias: the bare approximate one rounds with a
    // bias that adds up coherently over the layers a reflected flux crosses (1e-5 in scattering
    // bins)
    const float t2u = u * (2.0f - u);                                   // 1 - trans^2
    const float d = recip_nr(fmaf(b.c2, t2u, 1.0f));
    Ts = tr * d;
    Rs = b.qo * t2u * d;
    const float md = d * fmaf(-b.q, u, 1.0f + b.q);
    // isothermal (eq. 11): dB (1 - (1 - Ts + Rs)/2); otherwise eq. (15): cl phi dB (1 - Ts + Rs)/u
    Ss = dB * (iso ? fmaf(-b.hoh * md, u, 1.0f) : b.clh * phi * md);
    if constexpr (WANT_E) *Es = eo * u * fmaf(-b.q, tr, 1.0f) * d;
}

// (Ts, Rs, Ss) of the M sublayers of lane `sub` of a column (sublayer s between points s and
// s + 1; opacity the mean of the two points', Sect. 2.3, eq. 19) for a bin of kind KIND, and the
// product Ap of their transmissions.  Padding slots (zero opacity, column mass and Planck
// difference) take the zero-thickness form (1, 0, 0)
template <int KIND, int M>
__device__ __forceinline__ void coef_chunk(const BinConst& bc, const float* krow, const float* dm, const float* dbt,
                                           int sub, float dtau_iso, float (&Ts)[M], float (&Rs)[M], float (&Ss)[M],
                                           float& Ap)
{
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const int s = sub * M + k;
        const float dtau = 0.5f * (krow[s] + krow[s + 1]) * dm[s];
        layer_coef<false, false, KIND>(bc, dtau, dbt[s], dtau_iso, Ts[k], Rs[k], Ss[k]);
        Ap *= Ts[k];
    }
}

// ---------------------------------------------------------------------------
// 2^-floor(log2 m) for m > 0: scaling by it is exact (projective normalisation)
__device__ __forceinline__ float pow2_recip(float m)
{
    const int e = (__float_as_int(m) >> 23) & 0xff;
    return __int_as_float((254 - max(1, min(e, 253))) << 23);
}

// Exact solution of one column's coupled equations (the limit of the passes, Sect. 2.2.3) by
// the adding method, in deviation form.  With rho_s the reflectance of everything below point s
// (surface included: rho_0 = 1, since F_up,0 = F_dn,0 + pi B_int) and u_s the upward deviation
// that stack emits, G_up,s = rho_s G_dn,s + u_s and, per sublayer s,
//     kappa_s = 1 / (1 - Rs rho_s),  rho_{s+1} = Rs + Ts^2 rho_s kappa_s,
//     u_{s+1} = Ts kappa_s (u_s - rho_s Ss) + Ss,  G_dn,s = kappa_s (Ts G_dn,s+1 + Rs u_s - Ss).
// rho is carried in homogeneous coordinates (rho_h, sigma_h), rho = rho_h / (rho_h + sigma_h),
// sigma = 1 - rho, with the sublayer absorption Es = 1 - Ts - Rs.  Using Ts + Rs + Es = 1 the
// recurrence becomes the linear map
//     rho_h' = a rho_h + Rs sigma_h,  sigma_h' = b rho_h + (Ts + Es) sigma_h,
//     a = Ts (Ts + Rs) + Rs Es,  b = Es (2 Ts + Es),
// whose entries are all non-negative: neither rho nor 1 - rho is formed by a difference, for
// conservative scattering over the reflecting surface (rho = 1) as for an absorbing column
// (rho small); with rho_h + sigma_h = 1 the new sum is 1 - Rs rho = 1/kappa.  Each of the three
// recurrences (rho up, u up, G_dn down) is a warp scan: lane-local composition of its M
// sublayers, five shuffle levels (2x2 non-negative matrices, rescaled by powers of two, for rho;
// affine maps for u and G_dn), lane-local application.  Outputs per point lane*M + k:
// U[k] = G_up, Dn[k] = G_dn.
template <int M>
__device__ __forceinline__ void direct_column(const float (&Ts)[M], const float (&Rs)[M], const float (&Es)[M],
                                              const float (&Ss)[M], float (&U)[M], float (&Dn)[M], float toa_g,
                                              float bint, int lane)
{
    // (i) (rho_h, sigma_h), upwards from (1, 0)
    float p00 = 1.0f, p01 = 0.0f, p10 = 0.0f, p11 = 1.0f;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const float a = fmaf(Ts[k], Ts[k] + Rs[k], Rs[k] * Es[k]), b = Es[k] * fmaf(2.0f, Ts[k], Es[k]);
        const float r = Rs[k], d = Ts[k] + Es[k];
        const float n00 = fmaf(a, p00, r * p10), n01 = fmaf(a, p01, r * p11);
        const float n10 = fmaf(b, p00, d * p10), n11 = fmaf(b, p01, d * p11);
        p00 = n00; p01 = n01; p10 = n10; p11 = n11;
    }
    {
        const float sc = pow2_recip(fmaxf(fmaxf(p00, p01), fmaxf(p10, p11)));
        p00 *= sc; p01 *= sc; p10 *= sc; p11 *= sc;
    }
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
        const int dd = 1 << lv;
        const float q00 = __shfl_up_sync(FULL, p00, dd), q01 = __shfl_up_sync(FULL, p01, dd);
        const float q10 = __shfl_up_sync(FULL, p10, dd), q11 = __shfl_up_sync(FULL, p11, dd);
        if (lane >= dd) {                                   // P <- P . Q (the lanes below act first)
            const float n00 = fmaf(p00, q00, p01 * q10), n01 = fmaf(p00, q01, p01 * q11);
            const float n10 = fmaf(p10, q00, p11 * q10), n11 = fmaf(p10, q01, p11 * q11);
            const float sc = pow2_recip(fmaxf(fmaxf(n00, n01), fmaxf(n10, n11)));
            p00 = n00 * sc; p01 = n01 * sc; p10 = n10 * sc; p11 = n11 * sc;
        }
    }
    float rh, sh;
    {
        const float x = __shfl_up_sync(FULL, p00, 1), y = __shfl_up_sync(FULL, p10, 1);   // P_below (1, 0)
        const float inv = __frcp_rn(x + y);
        rh = lane == 0 ? 1.0f : x * inv;
        sh = lane == 0 ? 0.0f : y * inv;
    }
    float rho[M], kap[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const float a = fmaf(Ts[k], Ts[k] + Rs[k], Rs[k] * Es[k]), b = Es[k] * fmaf(2.0f, Ts[k], Es[k]);
        const float d = Ts[k] + Es[k];
        rho[k] = rh;
        kap[k] = __frcp_rn(fmaf(d, rh, sh));
        const float rn = fmaf(a, rh, Rs[k] * sh) * kap[k];
        sh = fmaf(b, rh, d * sh) * kap[k];
        rh = rn;
    }
    // (ii) u, upwards from u_0 = pi B_int: u' = al u + be, al = Ts kappa, be = Ss (1 - al rho)
    float A = 1.0f, B = 0.0f;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const float al = Ts[k] * kap[k];
        B = fmaf(al, B, Ss[k] * fmaf(-al, rho[k], 1.0f));
        A *= al;
    }
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
        const int dd = 1 << lv;
        const float Ao = __shfl_up_sync(FULL, A, dd), Bo = __shfl_up_sync(FULL, B, dd);
        if (lane >= dd) { B = fmaf(A, Bo, B); A *= Ao; }
    }
    {
        const float Ae = __shfl_up_sync(FULL, A, 1), Be = __shfl_up_sync(FULL, B, 1);
        float uu = lane == 0 ? bint : fmaf(Ae, bint, Be);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            U[k] = uu;                                      // u at point lane*M + k (reused below)
            const float al = Ts[k] * kap[k];
            uu = fmaf(al, uu, Ss[k] * fmaf(-al, rho[k], 1.0f));
        }
    }
    // (iii) G_dn, downwards from the TOA: G_dn,s = al G_dn,s+1 + ga, ga = kappa (Rs u - Ss)
    A = 1.0f; B = 0.0f;
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
        const float al = Ts[k] * kap[k];
        B = fmaf(al, B, kap[k] * fmaf(Rs[k], U[k], -Ss[k]));
        A *= al;
    }
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
        const int dd = 1 << lv;
        const float Ao = __shfl_down_sync(FULL, A, dd), Bo = __shfl_down_sync(FULL, B, dd);
        if (lane + dd < 32) { B = fmaf(A, Bo, B); A *= Ao; }
    }
    const float Ae = __shfl_down_sync(FULL, A, 1), Be = __shfl_down_sync(FULL, B, 1);
    float dn = lane == 31 ? toa_g : fmaf(Ae, toa_g, Be);
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
        dn = fmaf(Ts[k] * kap[k], dn, kap[k] * fmaf(Rs[k], U[k], -Ss[k]));
        Dn[k] = dn;
        U[k] = fmaf(rho[k], dn, U[k]);                      // G_up = rho G_dn + u
    }
}

// dynamic shared memory of one sweep block (CL lanes per column, lane chunk M, W = CL M point
// slots, G Gauss points): FP64 accumulators [3][W/2], the per-column rows of opacities / weighted
// downward deviations and of weighted upward deviations [2][G][W + 1], four per-point rows [W],
// and the TOA value
__host__ __device__ constexpr size_t sweep_smem_bytes(int M, int G, int CL = 32)
{
    return 3 * (size_t)(CL * M / 2) * sizeof(double) +
           (2 * (size_t)G * (CL * M + 1) + 4 * (size_t)(CL * M) + 1) * sizeof(float);
}

// threads of a sweep block: the exact solve takes one warp per Gauss point; the iterated passes
// take one warp per two Gauss points -- with 16-lane columns both at once (lanes 0-15 and 16-31),
// with 32-lane columns one after the other
__host__ __device__ constexpr int sweep_block_threads(int G, bool direct)
{
    return direct ? 32 * G : 32 * ((G + 1) / 2);
}

// resident blocks per SM that a sweep kernel is compiled for (its register budget): 32-lane
// columns, iterated passes -- three 320-thread blocks (64 registers) up to lane chunk 9 (chunk 9
// spills some registers and still runs faster than two blocks at 96), two (96) beyond; the exact
// solve -- two 640-thread blocks (48 registers) up to chunk 7, one beyond
template <int M, bool DIRECT>
constexpr int sweep_minb()
{
    return DIRECT ? (M <= 7 ? 2 : 1) : (M <= 9 ? 3 : 2);
}

// ---------------------------------------------------------------------------
// one work item = (atmosphere, tile of bins); the whole block cooperates
// CL = 32: a warp per Gauss point (the exact solve: all at once; the passes: the block's warps
// take the Gauss points in rounds); CL = 16: two Gauss points per warp (lanes 0-15 and 16-31),
// half the scan levels and fewer padded slots per column, at twice the registers per lane
template <int M, bool DIRECT, int CL = 32>
__device__ __forceinline__ void sweep_item(const PlanDev& P, int item, const int* __restrict__ status, int n_passes,
                                           int warm_valid, float* __restrict__ Fup_toa, float* __restrict__ F_spec,
                                           unsigned char* smem_raw)
{
    static_assert(CL == 32 || (CL == 16 && !DIRECT), "16-lane columns: iterated passes only");
    constexpr int W = CL * M;               // point slots per column
    constexpr int KST = W + 1;              // row stride of the per-column smem rows
    constexpr int LV = CL == 32 ? 5 : 4;    // scan levels
    const int G = P.G;
    const int tid = threadIdx.x, lane = tid & 31;
    // the Gauss point of this thread's column in the first round, and the Gauss points a round
    // covers (the exact solve: every point in one round)
    const int g_first = CL == 32 ? tid >> 5 : 2 * (tid >> 5) + (lane >> 4);
    const int g_round = CL == 32 ? (int)(blockDim.x >> 5) : 2 * (int)(blockDim.x >> 5);
    const int sub = lane & (CL - 1);        // the lane's place in its column
    const int2 it = P.items[item];
    if (status && status[it.x] != 0) return;
    const AtmDesc ad = P.atms[it.x];
    const TabDesc td = P.tabs[ad.tab];
    const int n = ad.n, NP = 2 * n + 1, NS = 2 * n;
    const int l_begin = it.y * P.TB;
    const int l_end = min(l_begin + P.TB, ad.L);

    double* acc = reinterpret_cast<double*>(smem_raw);         // [3][n+1], n+1 <= W/2
    float* kap = reinterpret_cast<float*>(acc + 3 * (W / 2));  // [G][KST] opacities, then w_g G_dn per point
    float* upr = kap + G * KST;                                // [G][KST] w_g G_up per point
    float* bt = upr + G * KST;                                 // [W] 2 pi eps B at points
    float* dbs = bt + W;                                       // [W] warm-start shift B_old - B_new
    float* dbt = dbs + W;                                      // [W] 2 pi eps (B_a - B_b) per sublayer
    float* dm = dbt + W;                                       // [W] sublayer column mass
    float* bc_toa = dm + W;                                    // [1] TOA value in deviation form

    const int nthreads = blockDim.x;
    for (int t = tid; t < W; t += nthreads) dm[t] = t < NS ? P.dm[ad.sub_off + t] : 0.0f;
    for (int t = tid; t < 3 * (n + 1); t += nthreads) acc[t] = 0.0;
    const int p_first = tid / G, g_of = tid - p_first * G;     // gather mapping: consecutive g
    const int p_stride = nthreads / G;
    // float4 gather over four consecutive g when rows stay 16-byte aligned
    const bool vec4 = (G & 3) == 0;
    const int G4 = G >> 2;
    const int p4_first = vec4 ? tid / G4 : 0, g4_of = vec4 ? tid - p4_first * G4 : 0;
    const int p4_stride = vec4 ? nthreads / G4 : 1;
    const float* tab = td.kappa;
    // warm-start columns (none when the launch keeps no warm start: then nothing is stored)
    float* wbase = P.warm ? P.warm + ad.warm_off : nullptr;

    for (int l = l_begin; l < l_end; ++l) {
        // the next bin's inputs move into L2 while this bin is processed: its constants, the
        // table rows at every point's four corners (first and last element of each) and, with a
        // warm start, its columns' upward deviations (one contiguous block of G W floats)
        if (l + 1 < l_end) {
            if (tid == 0) prefetch_l2(P.bins + ad.bin_off + l + 1);
            // (every species table of a mixed opacity, eq. 34)
            for (int sp = 0; sp < max(1, ad.n_spec); ++sp) {
                const float* ts = ad.n_spec > 1 ? P.tabs[P.spec_tab[ad.spec_off + sp]].kappa : tab;
                const int lg1 = (l + 1) * G;
                for (int p = tid; p < NP; p += nthreads) {
                    const float* r = ts + P.row[ad.pt_off + p] + lg1;
                    const float* c[4] = {r, r + td.offP, r + td.offT, r + td.offP + td.offT};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        prefetch_l2(c[j]);
                        prefetch_l2(c[j] + G - 1);
                    }
                }
            }
            if (!DIRECT && warm_valid && wbase) {
                const float* wn = wbase + (long long)(l + 1) * G * W;
                for (int i = tid * 32; i < G * W; i += nthreads * 32) prefetch_l2(wn + i);
            }
        }
        const BinConst bc = P.bins[ad.bin_off + l];
        const bool emits = !(bc.flags & (BIN_GREY_DARK | BIN_PURE_SCAT | BIN_GREY_THERM));
        // ---- phase 1: per-point Planck values, per-sublayer Planck differences.  Each warp
        // takes 31 consecutive points plus, in lane 31, the first point of the next group, so a
        // lane reads the Planck value of the point above from its neighbour (no barrier and no
        // second evaluation; lane 31's value serves only that read) ...
        // (the last warps take them: the block's first threads hold one opacity-gather task more)
        const int pw_need = (W + 30) / 31, pw_off = max(0, (nthreads >> 5) - pw_need);
        for (int p0 = ((tid >> 5) - pw_off) * 31; (tid >> 5) >= pw_off && p0 < W; p0 += ((nthreads >> 5) - pw_off) * 31) {
            const int p = p0 + lane;
            const bool pt = p < NP;
            const int q = ad.pt_off + p;
            float B = 0.0f, sh = 0.0f, d = 0.0f, x = 0.0f;
            if (pt && (bc.flags & BIN_GREY_THERM)) {
                const float T = P.Tf[q], c = 2.0f * bc.E;           // 2 eps sigma T^4
                const float T2 = T * T;
                B = c * T2 * T2;
                if (warm_valid) {
                    const float dT = P.dT_step[q], To = T + dT;
                    sh = c * dT * (To + T) * (To * To + T2);
                }
                if (p < NS) {
                    const float Tb = P.Tf[q + 1];
                    d = c * P.dT_sub[ad.sub_off + p] * (T + Tb) * (T2 + Tb * Tb);
                }
            } else if (pt && emits && P.btab) {
                const float* row = P.btab + (long long)(ad.bin_off + l) * kTabNT;
                const float T = P.Tf[q];
                B = planck_tab(row, T);
                if (warm_valid) sh = planck_tab(row, T + P.dT_step[q]) - B;
            } else if (pt && emits) {
                B = planck_ff(bc, P.invT[q], x);
                if (warm_valid) {
                    // B_old - B_new = B_new (e^y - 1) / (1 - e^{-x_old}), y = x_new - x_old (x_old: the
                    // high part of the old exponent, as planck_ff forms it); the old Planck value
                    // itself only for a large change (rare once the iteration settles: a branch)
                    const float y = bc.xs * P.dinv_step[q];
                    if (fabsf(y) < 1.0f) {
                        const float xo = bc.xs * P.invT_old[q].x;
                        sh = B * __fdividef(em1(y), -em1(-xo));
                    } else {
                        float xo;
                        sh = planck_ff(bc, P.invT_old[q], xo) - B;
                    }
                }
            }
            const float Bb = __shfl_down_sync(FULL, B, 1);          // B of point p + 1
            if (lane < 31 && p < W) {
                if (pt && emits && p < NS) {
                    if (P.btab) {
                        d = B - Bb;                                 // tabulated values
                    } else {
                        // B_a - B_b = B_b (e^y - 1) / (1 - e^{-x_a}), y = x_b - x_a
                        const float y = bc.xs * P.dinv_sub[ad.sub_off + p];
                        d = fabsf(y) < 1.0f ? Bb * __fdividef(em1(y), -em1(-x)) : B - Bb;
                    }
                }
                if (p == NP - 1) bc_toa[0] = bc.toa - B;
                bt[p] = B;
                dbs[p] = sh;
                dbt[p] = d;
            }
        }
        // ... and the opacity gather, consecutive threads on consecutive g
        if (ad.n_spec > 1) {
            // eq. (34): kappa = sum_j X_j kappa_j over species tables sharing the (T, P) grid, so
            // the corner offsets and weights of a point serve every species.  The species in turn
            // (table and weight read once per bin), each thread adding species j to its own
            // entries, in the order j = 0, 1, ... (kappa = fma(X_j, kappa_j, kappa) from 0)
            for (int j = 0; j < ad.n_spec; ++j) {
                const float* tj = P.tabs[P.spec_tab[ad.spec_off + j]].kappa;
                const float xj = P.spec_w[ad.spec_off + j];
                if (vec4) {
                    const int lg = l * G + 4 * g4_of;
                    for (int p = p4_first; p < NP; p += p4_stride) {
                        const int q = ad.pt_off + p;
                        const float4 w = P.wq[q];
                        const float* r = tj + P.row[q] + lg;
                        const float4 k00 = __ldg(reinterpret_cast<const float4*>(r));
                        const float4 k10 = __ldg(reinterpret_cast<const float4*>(r + td.offP));
                        const float4 k01 = __ldg(reinterpret_cast<const float4*>(r + td.offT));
                        const float4 k11 = __ldg(reinterpret_cast<const float4*>(r + td.offP + td.offT));
                        float* dst = kap + (4 * g4_of) * KST + p;
                        const float b0 = fmaf(w.w, k11.x, fmaf(w.z, k01.x, fmaf(w.y, k10.x, w.x * k00.x)));
                        const float b1 = fmaf(w.w, k11.y, fmaf(w.z, k01.y, fmaf(w.y, k10.y, w.x * k00.y)));
                        const float b2 = fmaf(w.w, k11.z, fmaf(w.z, k01.z, fmaf(w.y, k10.z, w.x * k00.z)));
                        const float b3 = fmaf(w.w, k11.w, fmaf(w.z, k01.w, fmaf(w.y, k10.w, w.x * k00.w)));
                        dst[0] = fmaf(xj, b0, j ? dst[0] : 0.0f);
                        dst[KST] = fmaf(xj, b1, j ? dst[KST] : 0.0f);
                        dst[2 * KST] = fmaf(xj, b2, j ? dst[2 * KST] : 0.0f);
                        dst[3 * KST] = fmaf(xj, b3, j ? dst[3 * KST] : 0.0f);
                    }
                } else {
                    const int lg = l * G + g_of;
                    for (int p = p_first; p < NP; p += p_stride) {
                        const int q = ad.pt_off + p;
                        float* dst = kap + g_of * KST + p;
                        *dst = fmaf(xj, kappa_at(tj, td, P.row[q], P.wq[q], lg), j ? *dst : 0.0f);
                    }
                }
            }
        } else if (vec4) {
            const int lg = l * G + 4 * g4_of;
            for (int p = p4_first; p < NP; p += p4_stride) {
                const int q = ad.pt_off + p;
                const float4 w = P.wq[q];
                const float* r = tab + P.row[q] + lg;
                const float4 k00 = __ldg(reinterpret_cast<const float4*>(r));
                const float4 k10 = __ldg(reinterpret_cast<const float4*>(r + td.offP));
                const float4 k01 = __ldg(reinterpret_cast<const float4*>(r + td.offT));
                const float4 k11 = __ldg(reinterpret_cast<const float4*>(r + td.offP + td.offT));
                float* dst = kap + (4 * g4_of) * KST + p;
                dst[0] = fmaf(w.w, k11.x, fmaf(w.z, k01.x, fmaf(w.y, k10.x, w.x * k00.x)));
                dst[KST] = fmaf(w.w, k11.y, fmaf(w.z, k01.y, fmaf(w.y, k10.y, w.x * k00.y)));
                dst[2 * KST] = fmaf(w.w, k11.z, fmaf(w.z, k01.z, fmaf(w.y, k10.z, w.x * k00.z)));
                dst[3 * KST] = fmaf(w.w, k11.w, fmaf(w.z, k01.w, fmaf(w.y, k10.w, w.x * k00.w)));
            }
        } else {
            const int lg = l * G + g_of;
            for (int p = p_first; p < NP; p += p_stride) {
                const int q = ad.pt_off + p;
                kap[g_of * KST + p] = kappa_at(tab, td, P.row[q], P.wq[q], lg);
            }
        }
        // the slots past the TOA point (KST - NP per column) hold zero opacity: with zero column mass
        // and Planck difference there, every padding sublayer takes the zero-thickness form (Ts = 1,
        // Rs = 0, Ss = 0) without a test per sublayer
        if (!DIRECT) {
            const int pad = KST - NP;
            for (int t = tid; t < G * pad; t += nthreads) kap[(t / pad) * KST + NP + t % pad] = 0.0f;
        }
        __syncthreads();

        // ---- phase 2: CL lanes per Gauss point; lane `sub` of a column holds its sublayers
        // sub*M .. sub*M+M-1 (the exact solve: CL = 32)
        if constexpr (DIRECT) {
            // the exact column solution (no passes, no warm start needed); a warp per Gauss point
            const int g = g_first;
            const float wg = P.gw[g];
            float Ts[M], Rs[M], Ss[M], Es[M], U[M], Dn[M];
            const float* krow = kap + g * KST;
            const float eo = __frcp_rn(1.0f + bc.q);               // 1 / (1 + q)
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const int s = lane * M + k;
                float t = 1.0f, r = 0.0f, src = 0.0f, e = 0.0f;
                if (s < NS) {
                    const float kabs = 0.5f * (krow[s] + krow[s + 1]);          // Sect. 2.3
                    if (bc.flags & BIN_RAYLEIGH) {
                        float kt;
                        const BinConst c = rayleigh_const(bc, P, kabs, kt);
                        layer_coef<true>(c, kt * dm[s], dbt[s], P.dtau_iso, t, r, src, &e,
                                         __frcp_rn(1.0f + c.q));
                    } else {
                        layer_coef<true>(bc, kabs * dm[s], dbt[s], P.dtau_iso, t, r, src, &e, eo);    // eq. (19)
                    }
                }
                Ts[k] = t;
                Rs[k] = r;
                Ss[k] = src;
                Es[k] = e;
            }
            const float toa_g = bc_toa[0];
            __syncwarp();                                           // the warp's row is free now
            direct_column<M>(Ts, Rs, Es, Ss, U, Dn, toa_g, bc.bint, lane);
            float* red_dn = kap + g * KST + lane * M;
            float* red_up = upr + g * KST + lane * M;
            // the warm start of later iterated passes, in their layout (CL' lanes per column, lane
            // chunk M'; point p at slot (p mod M') CL' + p / M').  At 32 lanes that is this warp's
            // own layout.  At 16 the column goes through the warp's shared-memory row first, so
            // that consecutive lanes write consecutive slots
            if (ad.cl == 32) {                  // (a plan always holds a warm-start buffer)
                const long long col = (long long)(l * G + g) * W;
#pragma unroll
                for (int k = 0; k < M; ++k) wbase[col + k * 32 + lane] = U[k];
            } else {
                const int wm = ad.M;
                const long long col = (long long)(l * G + g) * (16 * wm);
#pragma unroll
                for (int k = 0; k < M; ++k) red_up[k] = U[k];
                __syncwarp();
                const float* row = upr + g * KST;
                for (int i = lane; i < 16 * wm; i += 32) wbase[col + i] = row[(i & 15) * wm + (i >> 4)];
                __syncwarp();
            }
#pragma unroll
            for (int k = 0; k < M; ++k) {
                red_dn[k] = wg * Dn[k];
                red_up[k] = wg * U[k];
            }
        } else {
            // the Gauss points in rounds of g_round (the block holds a warp per two Gauss points:
            // one round of two columns per warp at CL = 16, two rounds at CL = 32; odd G: the last
            // warp idles in the last round, or its upper half does)
            constexpr int ROUNDS = CL == 16 ? 1 : 2;
#pragma unroll 1
            for (int r = 0; r < ROUNDS; ++r) {
                const int g_raw = r * g_round + g_first;
                const bool g_ok = g_raw < G;
                const int g = g_ok ? g_raw : G - 1;
                const float wg = g_ok ? P.gw[g] : 0.0f;
                float Ts[M], Rs[M], Ss[M], X[M + 1];
                float Ap = 1.0f;
                const float* krow = kap + g * KST;
                // initial upward deviation: previous evaluation shifted to the new Planck values, or
                // F_up = 0 (Sect. 2.2.3: the coupled stream starts from zero); loaded first, so that
                // the loads complete under the coefficients
                const long long col = (long long)(l * G + g) * W;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const int p = sub * M + k;
                    X[k] = (warm_valid && wbase) ? wbase[col + k * CL + sub] + dbs[p] : -bt[p];
                }
                X[M] = 0.0f;
                if (bc.flags & BIN_RAYLEIGH) {                                      // uniform per bin
#pragma unroll
                    for (int k = 0; k < M; ++k) {
                        const int s = sub * M + k;
                        float t, r, src;                                    // padding: (1, 0, 0)
                        float kt;
                        const BinConst c = rayleigh_const(bc, P, 0.5f * (krow[s] + krow[s + 1]), kt);
                        layer_coef(c, kt * dm[s], dbt[s], P.dtau_iso, t, r, src);
                        Ts[k] = t;
                        Rs[k] = r;
                        Ss[k] = src;
                        Ap *= t;
                    }
                } else if (P.utab) {                                                // uniform per launch
#pragma unroll
                    for (int k = 0; k < M; ++k) {
                        const int s = sub * M + k;
                        float t, r, src;                                    // padding: (1, 0, 0)
                        const float dtau = 0.5f * (krow[s] + krow[s + 1]) * dm[s];   // Sect. 2.3, eq. (19)
                        layer_coef<false, true>(bc, dtau, dbt[s], P.dtau_iso, t, r, src, nullptr, 0.0f, P.utab);
                        Ts[k] = t;
                        Rs[k] = r;
                        Ss[k] = src;
                        Ap *= t;
                    }
                } else if (bc.flags & BIN_PURE_SCAT) {                              // uniform per bin
                    coef_chunk<COEF_PURE_SCAT>(bc, krow, dm, dbt, sub, P.dtau_iso, Ts, Rs, Ss, Ap);
                } else if (bc.flags & BIN_NO_SCAT) {
                    coef_chunk<COEF_NO_SCAT>(bc, krow, dm, dbt, sub, P.dtau_iso, Ts, Rs, Ss, Ap);
                } else {
                    coef_chunk<COEF_GENERAL>(bc, krow, dm, dbt, sub, P.dtau_iso, Ts, Rs, Ss, Ap);
                }
                // scan multipliers (depend on the transmissions only)
                float adn[LV], aup[LV], adn_fin, aup_fin;
                {
                    float a = Ap;
#pragma unroll
                    for (int lv = 0; lv < LV; ++lv) {
                        const int d = 1 << lv;
                        const float ao = __shfl_down_sync(FULL, a, d, CL);
                        const bool ok = sub + d < CL;
                        adn[lv] = ok ? a : 0.0f;
                        a = ok ? a * ao : a;
                    }
                    adn_fin = a;
                    a = Ap;
#pragma unroll
                    for (int lv = 0; lv < LV; ++lv) {
                        const int d = 1 << lv;
                        const float ao = __shfl_up_sync(FULL, a, d, CL);
                        const bool ok = sub >= d;
                        aup[lv] = ok ? a : 0.0f;
                        a = ok ? a * ao : a;
                    }
                    aup_fin = a;
                }
                const float toa_g = bc_toa[0];
                const float bint = bc.bint;
                __syncwarp();
                // weighted deviations of every point of the column (phase 3 reads the interfaces);
                // the opacity row is free now
                float* red_dn = kap + g * KST + sub * M;
                float* red_up = upr + g * KST + sub * M;
                const int K = (bc.flags & BIN_NO_SCAT) ? 1 : n_passes;
                for (int pass = 0; pass < K; ++pass) {
                    const bool last = pass == K - 1;
                    // downward sweep: G_dn[s] = Ts G_dn[s+1] + (Rs G_up[s] - Ss), from the TOA
                    {
                        // G_up[s] enters only through Rs G_up[s] - Ss: X[k] is replaced by that term
                        float b = 0.0f;
#pragma unroll
                        for (int k = M - 1; k >= 0; --k) {
                            X[k] = fmaf(Rs[k], X[k], -Ss[k]);
                            b = fmaf(Ts[k], b, X[k]);
                        }
#pragma unroll
                        for (int lv = 0; lv < LV; ++lv) b = fmaf(adn[lv], __shfl_down_sync(FULL, b, 1 << lv, CL), b);
                        const float outv = fmaf(adn_fin, toa_g, b);
                        float inv = __shfl_down_sync(FULL, outv, 1, CL);
                        if (sub == CL - 1) inv = toa_g;
                        X[M] = inv;
#pragma unroll
                        for (int k = M - 1; k >= 0; --k) X[k] = fmaf(Ts[k], X[k + 1], X[k]);
                        if (last && g_ok) {
#pragma unroll
                            for (int k = 0; k < M; ++k) red_dn[k] = wg * X[k];
                        }
                    }
                    // upward sweep: G_up[s+1] = Ts G_up[s] + (Rs G_dn[s+1] + Ss), from the BOA (eq. 22)
                    {
                        // G_dn[s+1] enters only through Rs G_dn[s+1] + Ss: X[k+1] is replaced by that term
                        float c = 0.0f;
#pragma unroll
                        for (int k = 0; k < M; ++k) {
                            X[k + 1] = fmaf(Rs[k], X[k + 1], Ss[k]);
                            c = fmaf(Ts[k], c, X[k + 1]);
                        }
#pragma unroll
                        for (int lv = 0; lv < LV; ++lv) c = fmaf(aup[lv], __shfl_up_sync(FULL, c, 1 << lv, CL), c);
                        const float boa = __shfl_sync(FULL, X[0], 0, CL) + bint;
                        const float outv = fmaf(aup_fin, boa, c);
                        float inv = __shfl_up_sync(FULL, outv, 1, CL);
                        if (sub == 0) inv = boa;
                        X[0] = inv;
#pragma unroll
                        for (int k = 0; k < M; ++k) X[k + 1] = fmaf(Ts[k], X[k], X[k + 1]);
                        if (last && g_ok) {
#pragma unroll
                            for (int k = 0; k < M; ++k) red_up[k] = wg * X[k];
                        }
                    }
                }
                if (g_ok && wbase) {
#pragma unroll
                    for (int k = 0; k < M; ++k) wbase[col + k * CL + sub] = X[k];
                }
            }
        }
        __syncthreads();
        // optional per-bin fluxes at every point (a debug output): sum_g w_g G + 2 pi eps B in
        // double, fixed order; [up points 0..2n][down points 0..2n] per bin
        if (F_spec) {
            float* fs = F_spec + ad.fspec_off + (long long)l * 2 * NP;
            for (int t = tid; t < 2 * NP; t += nthreads) {
                const bool up = t < NP;
                const int q = up ? t : t - NP;
                const float* row = (up ? upr : kap) + q;
                double sg = 0.0;
                for (int gg = 0; gg < G; ++gg) sg += (double)row[gg * KST];
                fs[t] = (float)(sg + (double)bt[q]);
            }
        }
        // ---- phase 3: Gauss-point sums (fixed order, float) into the item's FP64 accumulators.
        // Thread t sums interface t's column of the per-warp rows (downward interfaces 0..n, then
        // upward interfaces 0..n; interface i is point 2i); the threads after them add the Planck
        // fluxes at the interfaces
        const int NI = n + 1;
        for (int t = tid; t < 3 * NI; t += nthreads) {
            if (t == 2 * NI - 1) continue;                 // TOA upward: summed below
            double v;
            int a;
            if (t < 2 * NI) {
                const bool dn = t < NI;
                const float* row = (dn ? kap : upr) + 2 * (dn ? t : t - NI);
                float sg = 0.0f;
                for (int gg = 0; gg < G; ++gg) sg += row[gg * KST];
                v = (double)sg;
                a = dn ? NI + t : t - NI;
            } else {
                v = (double)bt[2 * (t - 2 * NI)];
                a = t;
            }
            acc[a] += v;
        }
        // the emergent bin: sum_g w_g G_up(TOA) as a float-float reduction over the lanes of the
        // last warp (error-free sums in a fixed butterfly), then the Planck add-back in double
        if (tid >= nthreads - 32) {
            float2 sv = make_float2(lane < G ? upr[lane * KST + NS] : 0.0f, 0.0f);
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) {
                const float2 o = make_float2(__shfl_xor_sync(FULL, sv.x, d), __shfl_xor_sync(FULL, sv.y, d));
                sv = ff_add(sv, o);
            }
            if (lane == 0) {
                const double sud = (double)sv.x + (double)sv.y;
                if (Fup_toa) Fup_toa[ad.bin_off + l] = (float)(sud + (double)bt[2 * n]);
                acc[n] += sud;
            }
        }
        __syncthreads();
    }
    double* part = P.part + ad.part_off + (long long)it.y * 3 * (n + 1);
    for (int t = tid; t < 3 * (n + 1); t += nthreads) part[t] = acc[t];
}

// counter == nullptr: block b takes item order[b].  Otherwise persistent: the resident
// blocks pull items (in cost order) from counter[0] until the group is exhausted; counter[1]
// counts the blocks that have left, and the last one to leave returns both to zero for the
// next launch (every block has then stopped pulling), so no reset is needed between launches.
template <int M, int MINB, bool DIRECT = false, int CL = 32>
__global__ void __launch_bounds__(sweep_block_threads(20, DIRECT), MINB)
    sweep_kernel(PlanDev P, const int* __restrict__ order, int count, int* __restrict__ counter,
                 const int* __restrict__ status, int n_passes, int warm_valid, float* __restrict__ Fup_toa,
                 float* __restrict__ F_spec)
{
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (!counter) {
        sweep_item<M, DIRECT, CL>(P, order[blockIdx.x], status, n_passes, warm_valid, Fup_toa, F_spec, smem_raw);
        return;
    }
    __shared__ int s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int k = s_next;
        if (k >= count) break;
        sweep_item<M, DIRECT, CL>(P, order[k], status, n_passes, warm_valid, Fup_toa, F_spec, smem_raw);
        __syncthreads();                    // shared memory is reused by the next item
    }
    if (threadIdx.x == 0 && atomicAdd(counter + 1, 1) == (int)gridDim.x - 1) {
        atomicExch(counter, 0);
        atomicExch(counter + 1, 0);
    }
}

// ---------------------------------------------------------------------------
// bolometric fluxes, one warp per interface: F_up = sum_items (sum G_up + sum B),
// F_dn likewise; lane-strided FP64 sums and a fixed xor-shuffle tree (deterministic)
// interface i's bolometric fluxes by one warp: lane-strided fixed-order FP64 sums over the
// atmosphere's work items and a fixed xor tree (deterministic)
__device__ __forceinline__ void finalize_sums(const PlanDev& P, const AtmDesc& ad, int i, int lane, double& up,
                                              double& dn)
{
    const int n = ad.n, stride = 3 * (n + 1);
    const double* part = P.part + ad.part_off;
    double su = 0.0, sd = 0.0, sb = 0.0;
#pragma unroll 4
    for (int t = lane; t < ad.n_items; t += 32) {
        su += part[t * stride + i];
        sd += part[t * stride + (n + 1) + i];
        sb += part[t * stride + 2 * (n + 1) + i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(FULL, su, o);
        sd += __shfl_xor_sync(FULL, sd, o);
        sb += __shfl_xor_sync(FULL, sb, o);
    }
    up = su + sb;
    dn = sd + sb;
}

__global__ void finalize_kernel(PlanDev P, const int* __restrict__ status, double* __restrict__ Fup,
                                double* __restrict__ Fdn)
{
    pdl_enter();
    const int a = blockIdx.y;
    if (status && status[a] != 0) return;
    const AtmDesc ad = P.atms[a];
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i > ad.n) return;
    double up, dn;
    finalize_sums(P, ad, i, lane, up, dn);
    if (lane == 0) {
        Fup[ad.if_off + i] = up;
        Fdn[ad.if_off + i] = dn;
    }
}

// ---------------------------------------------------------------------------
// temperature step, eqs. (23)-(29), FP64
struct TempArgs {
    double sigma, tol, fpre_num, fpre_exp, osc_down, osc_up, mult_max, T_floor;
    double T_tab_max;       // > 0: the top of the tabulated Planck range (Sect. 2.6 tables); a layer above
                            // it ends the atmosphere as OUT_OF_RANGE
    int max_iter;
};

__device__ __forceinline__ double layer_divergence(const double* fu, const double* fd, int i)
{
    return (fu[i + 1] - fd[i + 1]) - (fu[i] - fd[i]);
}

// metric (eq. 29) and temperature step (eqs. 23-28, Sect. 2.2.4) of atmosphere a by one block
// (blockDim >= n, a multiple of 32; every thread of the block calls it): the block reduces the
// metric itself, so no separate reduction launch and no atomics are needed.  Fu, Fd: the
// atmosphere's bolometric fluxes at its n+1 interfaces (global or shared memory).
__device__ __forceinline__ void temp_block(const PlanDev& P, const TempArgs& targ, const AtmDesc& ad, int a,
                                           const double* Fu, const double* Fd, double* __restrict__ T_layer,
                                           double* __restrict__ mult, uint8_t* __restrict__ hist,
                                           uint8_t* __restrict__ nhist, int* __restrict__ status,
                                           int* __restrict__ iters, double* __restrict__ metric_out,
                                           int* __restrict__ n_active, unsigned long long* s_max)
{
    const int i = threadIdx.x, lane = i & 31, w = i >> 5;
    const bool mine = i < ad.n;
    const int li = ad.lay_off + i;
    double dF = 0.0, Ti = 1.0, m_old = 1.0, step = 0.0;
    unsigned h_old = 0u, c_old = 0u;
    unsigned long long bits = 0ull;
    if (mine) {
        // the layer's state and its candidate step are read and formed before the block-wide
        // reduction (no barrier in between, so the loads and the FP64 pow overlap it); they are
        // applied below only while the atmosphere is not converged
        m_old = mult[li];
        h_old = hist[li];
        c_old = nhist[li];
        const double lnr = P.lnr[li];
        dF = layer_divergence(Fu, Fd, i);
        Ti = T_layer[li];
        double m = fabs(dF) / (targ.sigma * Ti * Ti * Ti * Ti);
        if (!(m == m) || !isfinite(Ti) || isinf(m)) m = __longlong_as_double(0x7ff8000000000000ll);
        bits = (unsigned long long)__double_as_longlong(m);
        if (dF != 0.0) {
            const double mag = targ.fpre_num * pow(fabs(dF), 1.0 - targ.fpre_exp) / (targ.sigma * Ti * Ti * Ti * lnr);
            step = -m_old * (dF > 0.0 ? mag : -mag);
        }
    }
    // non-negative doubles order like their bit patterns (NaN above +inf): an exact max
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, bits, d);
        bits = o > bits ? o : bits;
    }
    if (lane == 0) s_max[w] = bits;
    __syncthreads();
    if (w == 0) {
        bits = lane < (int)(blockDim.x >> 5) ? s_max[lane] : 0ull;
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, bits, d);
            bits = o > bits ? o : bits;
        }
        if (lane == 0) s_max[0] = bits;
    }
    __syncthreads();
    const double worst = __longlong_as_double((long long)s_max[0]);
    const bool bad = !(worst == worst);
    if (i == 0) {
        const int itn = (iters ? iters[a] : 0) + 1;
        if (iters) iters[a] = itn;
        if (metric_out) metric_out[a] = worst;
        int st = 0;
        if (bad) st = 3;
        else if (worst < targ.tol) st = 1;
        else if (itn >= targ.max_iter) st = 2;
        if (st) {
            status[a] = st;
            if (n_active) atomicSub(n_active, 1);
        }
    }
    if (mine && !bad && !(worst < targ.tol)) {
        double Tn = Ti + step;
        if (Tn < targ.T_floor) Tn = targ.T_floor;
        T_layer[li] = Tn;
        const unsigned h = (h_old << 1 | (step > 0.0 ? 1u : 0u)) & 0x3Fu;
        hist[li] = (uint8_t)h;
        unsigned c = c_old;
        if (c < 6) c += 1;
        nhist[li] = (uint8_t)c;
        if (c >= 6) {
            double m = m_old;
            if (h == 0u || h == 0x3Fu) m = fmin(m * targ.osc_up, targ.mult_max);
            else m = m * targ.osc_down;
            mult[li] = m;
        }
    }
    if (targ.T_tab_max > 0.0) {
        // with tabulated Planck functions, a temperature above the table's last node would take
        // that node's values: the atmosphere stops with its own status instead
        const int out = __syncthreads_or(mine && !(T_layer[li] <= targ.T_tab_max));
        if (out && i == 0 && status[a] == 0) {
            status[a] = 4;
            if (n_active) atomicSub(n_active, 1);
        }
    }
}

__global__ void temp_kernel(PlanDev P, TempArgs targ, const double* __restrict__ Fup, const double* __restrict__ Fdn,
                            double* __restrict__ T_layer, double* __restrict__ mult, uint8_t* __restrict__ hist,
                            uint8_t* __restrict__ nhist, int* __restrict__ status, int* __restrict__ iters,
                            double* __restrict__ metric_out, int* __restrict__ n_active)
{
    __shared__ unsigned long long s_max[32];
    const int a = blockIdx.x;
    if (status[a] != 0) return;
    const AtmDesc ad = P.atms[a];
    temp_block(P, targ, ad, a, Fup + ad.if_off, Fdn + ad.if_off, T_layer, mult, hist, nhist, status, iters,
               metric_out, n_active, s_max);
}

constexpr int kPostMaxIf = 256;     // interfaces of the deepest supported atmosphere (239 layers)

// Everything after the sweep of one RE step, one block per atmosphere: the bolometric fluxes
// (finalize_sums), the metric and temperature step (temp_block), and, with do_prep, the point
// quantities of the next evaluation at the new temperatures (prep_point with the warm-start
// shift) -- so an iteration inside helios_solve_re is two launches: sweep and this.
// gate: atmospheres whose status is not ACTIVE are skipped (inside helios_solve_re); without it
// every atmosphere is stepped and its status recomputed (helios_re_step).  do_finalize: the
// bolometric sums are done here (few work items per atmosphere); otherwise finalize_kernel,
// spread over many blocks, has written Fup/Fdn already.
__global__ void post_kernel(PlanDev P, TempArgs targ, double* __restrict__ Fup, double* __restrict__ Fdn,
                            double* __restrict__ T_layer, double* __restrict__ mult, uint8_t* __restrict__ hist,
                            uint8_t* __restrict__ nhist, int* __restrict__ status, int* __restrict__ iters,
                            double* __restrict__ metric_out, int* __restrict__ n_active, int gate, int do_finalize,
                            int do_prep)
{
    pdl_enter();
    __shared__ double sF[2][kPostMaxIf];
    __shared__ unsigned long long s_max[32];
    const int a = blockIdx.x;
    if (gate && status[a] != 0) return;
    if (!gate && threadIdx.x == 0) status[a] = 0;   // re-decided by this step's metric
    const AtmDesc ad = P.atms[a];
    const double* Fu = Fup + ad.if_off;
    const double* Fd = Fdn + ad.if_off;
    if (do_finalize) {
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int i = threadIdx.x >> 5; i <= ad.n; i += nw) {
            double up, dn;
            finalize_sums(P, ad, i, lane, up, dn);
            if (lane == 0) {
                Fup[ad.if_off + i] = up;
                Fdn[ad.if_off + i] = dn;
                sF[0][i] = up;
                sF[1][i] = dn;
            }
        }
        Fu = sF[0];
        Fd = sF[1];
    }
    __syncthreads();
    temp_block(P, targ, ad, a, Fu, Fd, T_layer, mult, hist, nhist, status, iters, metric_out, n_active, s_max);
    if (!do_prep) return;
    __syncthreads();                        // the new temperatures and the status are visible
    if (status[a] != 0) return;             // converged or failed in this step: no next evaluation
    for (int p = threadIdx.x; p < 2 * ad.n + 1; p += blockDim.x) prep_point(P, T_layer, ad, p, 1);
}

// ---------------------------------------------------------------------------
// standalone opacity interpolation (same coordinate, corner and weight code as the fused path)
__global__ void interp_kernel(PlanDev P, const double* __restrict__ T_layer, int a, float* __restrict__ kappa_out,
                              long long kap_off, int32_t* __restrict__ idx_out, double* __restrict__ w_out)
{
    const AtmDesc ad = P.atms[a];
    const TabDesc td = P.tabs[ad.tab];
    const int n = ad.n, np = 2 * n + 1;
    const double* T = T_layer + ad.lay_off;
    const long long total = (long long)np * ad.L * P.G;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < total;
         f += (long long)gridDim.x * blockDim.x) {
        const int g = (int)(f % P.G);
        const long long pl = f / P.G;
        const int l = (int)(pl % ad.L);
        const int p = (int)(pl / ad.L);
        const int q = ad.pt_off + p;
        int it, row;
        double wt;
        float4 wq;
        table_coord(point_T(T, n, p, P.iso_layers), td.T0, td.dT, td.nT, it, wt);
        point_corners(td, P.iP[q], P.wP[q], it, wt, row, wq);
        if (kappa_out) {
            float k;
            if (ad.n_spec > 1) {
                k = 0.0f;
                for (int j = 0; j < ad.n_spec; ++j)
                    k = fmaf(P.spec_w[ad.spec_off + j], kappa_at(P.tabs[P.spec_tab[ad.spec_off + j]].kappa, td, row, wq,
                                                                 l * P.G + g), k);
            } else {
                k = kappa_at(td.kappa, td, row, wq, l * P.G + g);
            }
            kappa_out[kap_off + f] = k;
        }
        if (l == 0 && g == 0) {
            if (idx_out) { idx_out[2 * q] = P.iP[q]; idx_out[2 * q + 1] = it; }
            if (w_out) { w_out[2 * q] = P.wP[q]; w_out[2 * q + 1] = wt; }
        }
    }
}

}  // namespace helios_dev
