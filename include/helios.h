/*
 * helios.h -- C ABI of the B300-native radiative-equilibrium hot path of
 * HELIOS (Malik et al. 2016, arXiv:1606.05474).
 *
 * Conventions shared by every call
 * --------------------------------
 * Units are CGS (erg, cm, g, s, K); pressures are given in bar.
 * An atmosphere has n layers (layer 0 at the bottom), n+1 interfaces
 * (interface 0 = BOA, interface n = TOA; Sect. 2.2.1, Fig. 2) and, with the
 * non-isothermal two-sublayer grid, 2n+1 points (point 2i = interface i,
 * point 2i+1 = centre of layer i).
 * A batch holds A atmospheres with their own layer and bin counts.  Per-layer
 * arrays are packed atmosphere after atmosphere: atmosphere a starts at
 * sum_{b<a} n_b (layers), sum_{b<a} (n_b+1) (interfaces), sum_{b<a} L_b
 * (bins), sum_{b<a} (2 n_b + 1) (points).
 *
 * Memory ownership: pointers documented "host" are read during the call only.
 * Pointers documented "device" are caller-owned device memory on the plan's
 * device; the library never frees them.  The library allocates only its
 * context, its plans and each plan's internal workspace (helios_plan_create).
 *
 * Streams: every compute call is asynchronous on the given CUDA stream and
 * returns before the GPU work completes, except helios_solve_re, which
 * synchronises (it reads back the number of atmospheres still iterating).
 *
 * Errors: every call returns HELIOS_OK (0) or a negative code; the message of
 * the last failure on the calling thread is returned by helios_last_error().
 * The library never aborts, traps or prints.  Invalid arguments are rejected
 * before any GPU work is queued.
 */
#ifndef HELIOS_H
#define HELIOS_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HELIOS_VERSION 100

enum {
    HELIOS_OK = 0,
    HELIOS_EINVAL = -1,     /* bad shape, pointer or parameter */
    HELIOS_ENOMEM = -2,     /* workspace allocation failed */
    HELIOS_ECUDA = -3,      /* a CUDA call failed (message in helios_last_error) */
    HELIOS_ENOCONV = -5     /* helios_solve_re: some atmosphere did not converge (see status[]) */
};

/* n_passes value of helios_flux_sweep: instead of a number of scattering passes, solve each
 * column's coupled two-stream equations exactly -- the limit the passes of Sect. 2.2.3
 * approach (the adding method, warp-parallel; fluxes then do not depend on a warm start). */
#define HELIOS_DIRECT (-1)

/* Per-atmosphere status of the radiative-equilibrium iteration. */
enum {
    HELIOS_ATM_ACTIVE = 0,        /* still iterating */
    HELIOS_ATM_CONVERGED = 1,     /* eq. (29) holds in every layer */
    HELIOS_ATM_NOT_CONVERGED = 2, /* hit max_iter */
    HELIOS_ATM_NONFINITE = 3,     /* a non-finite flux or temperature appeared; frozen */
    HELIOS_ATM_OUT_OF_RANGE = 4   /* params.tabulate: a temperature left the tabulated Planck range
                                     (above 6000 K); frozen */
};

typedef struct helios_ctx helios_ctx;
typedef struct helios_plan helios_plan;

/* Correlated-k table (Sect. 2.3): kappa[nP][nT][L][G] in cm^2/g (device,
 * float32, 16-byte aligned), tabulated at log10 P[bar] = log10P0 + i*dlog10P
 * and T[K] = T0 + j*dT.  Interpolated bilinearly in (T, log10 P) and clamped
 * to the nearest tabulated value outside the table (Sect. 2.3, footnote).
 * G is the number of Gauss-Legendre points per bin (1 <= G <= 32); the
 * table's g index runs over the Gauss-Legendre nodes of [0, 1] in ascending
 * order (eqs. 30-32).  All tables of a plan share one G. */
typedef struct {
    int nP, nT, L, G;
    double log10P0, dlog10P, T0, dT;
    const float* kappa;
} helios_ktable_t;

/* A batch of atmospheres (all arrays host, read by helios_plan_create only).
 * Atmosphere a: n_layers[a] >= 2 layers whose centres are log-spaced from
 * P_bot_bar[a] (bottom) to P_top_bar[a] (top) (Sect. 2.2.1, Sect. 3);
 * n_bins[a] >= 1 wavelength bins with edges nu_edges (cm^-1, increasing,
 * n_bins[a]+1 values, packed); per-bin single-scattering albedo omega0 and
 * asymmetry factor g0 (packed, n_bins[a] values, Sect. 2.1.1); it uses bins
 * 0..n_bins[a]-1 of table table_id[a].  grav: cm s^-2.  T_irr: the incident
 * diffuse stellar flux is sigma*T_irr^4, spread over the bins like a
 * blackbody at T_star (Sect. 2.2.2, eq. 20, with f (R_star/a)^2 folded into
 * T_irr).  T_int: the internal flux sigma*T_int^4 enters at the BOA, spread
 * like a blackbody at T_int (eqs. 21-22). */
typedef struct {
    int A;
    const int32_t* n_layers;
    const int32_t* n_bins;
    const int32_t* table_id;
    const double* P_top_bar;
    const double* P_bot_bar;
    const double* grav;
    const double* T_irr;
    const double* T_int;
    const double* T_star;
    const double* nu_edges;
    const float* omega0;
    const float* g0;
    /* Optional species mixing (Sect. 2.3, eqs. 34-35): when species_off is not NULL,
     * atmosphere a's opacity is sum_j species_weight[j] * kappa_{species_table[j]}
     * over j in [species_off[a], species_off[a+1]) (mass mixing ratios times the
     * species' k-tables, perfectly correlated as in the paper); every table of an
     * atmosphere must share its (T, P) grid, L and G; at most 16 species.  NULL:
     * the single table table_id[a] with weight 1. */
    const int32_t* species_off;     /* [A+1] or NULL */
    const int32_t* species_table;
    const double* species_weight;
} helios_batch_t;

/* Method parameters; helios_default_params fills the paper's values. */
typedef struct {
    double D;            /* diffusivity factor, eps = 1/D (Sect. 3: 2) */
    double dtau_iso;     /* sublayers thinner than this use the isothermal form (Sect. 2.2.1: 1e-4) */
    double w0_pure;      /* 1 - omega0 below this uses the pure-scattering form (Sect. 2.1.4: 1e-6) */
    double tol;          /* convergence: |dF_i|/(sigma T_i^4) < tol in every layer (eq. 29: 1e-7) */
    double fpre_num;     /* f_pre = fpre_num / |dF|^fpre_exp (eq. 28: 1e5, 0.9) */
    double fpre_exp;
    double osc_down;     /* timestep factor after an oscillation (Sect. 2.2.4: 0.67) */
    double osc_up;       /* timestep factor after a monotonic run (Sect. 2.2.4: 1.1) */
    double mult_max;     /* cap on the per-layer timestep multiplier (10; the paper states none) */
    double T_floor;      /* temperatures are kept >= T_floor (1 K) */
    int n_scat;          /* extra scattering passes per temperature step (Sect. 2.2.3: 4) */
    int max_iter;        /* helios_solve_re: maximum flux evaluations per atmosphere */
    int grey_mode;       /* 1: two-bin grey test mode (bin 0 visible: no emission, all stellar flux;
                            bin 1 thermal: pi*B = sigma T^4, all internal flux) */
    int printed_gradient;/* 1: gradient prefactor eps/(1 + w0 g0) as printed in eq. (15) */
    int bins_per_item;   /* bins one thread block processes per work item (0: automatic) */
    int check_every;     /* helios_solve_re: iterations per CUDA-graph launch between checks (0: auto) */
    int persistent;      /* 1: a resident grid pulls work items from a counter; 0: one block per item */
    int iso_layers;      /* 0: non-isothermal layers, two linear-B sublayers each (Sect. 2.2.1, Fig. 2);
                            1: isothermal layers (Sect. 2.2.1, eqs. 9, 11): layer i at its centre
                            temperature and pressure, opacity at the centre, optical thickness over
                            the whole layer -- the grid of the emission spectra computed as a
                            post-processing step (Sect. 3; with n_passes = 81, Sect. 2.2.3) */
    int device_loop;     /* helios_solve_re: 1: the whole iteration is one CUDA graph whose conditional
                            WHILE node repeats check_every steps until no atmosphere is active (no host
                            round trip); 0: the host relaunches a graph of check_every steps and reads
                            the active count in between */
    int direct;          /* 1: evaluations with the plan's default passes (n_passes = 0, and every step
                            of helios_solve_re) solve each column's coupled equations exactly instead of
                            making 1 + n_scat passes (HELIOS_DIRECT below) */
    int rayleigh;        /* 1: Rayleigh scattering by H2 (Sect. 2.1.4, eqs. 16-17): its opacity, per
                            bin at the bin's centre wavelength over mbar = 2.4 m_p, joins every
                            sublayer's opacity, and omega0 = kappa_R / (kappa + kappa_R) per sublayer,
                            bin and g (the batch's omega0 is then not used; g0 is) */
    int col_lanes;       /* lanes per column of the iterated sweep: 32 (one warp per Gauss point), 16
                            (two Gauss points per warp: fewer scan steps and padded sublayer slots
                            per column, twice the registers per lane; atmospheres of 24 to 119
                            layers, others are rejected), or 0: 16 where an atmosphere has 24 to 119
                            layers, else 32.  Results agree to rounding; the exact column solve
                            always runs 32 lanes per column */
    int tabulate;        /* 1: the Planck and transmission functions come from tables (Sect. 2.6):
                            each bin's Planck flux at 10 K nodes, linear in T between them, and
                            1 - e^-x of the layer exponent x = lambda dtau at nodes 0.1 apart in
                            log10 x, linear in x between them (x below 10^-8.05, 1 above 10^2.05).
                            Not with iso_layers, direct, rayleigh or grey_mode, nor with
                            n_passes = HELIOS_DIRECT; holds bins x 601 floats of device memory */
} helios_params_t;

void helios_default_params(helios_params_t* p);
int helios_version(void);
const char* helios_last_error(void);

/* Context on CUDA device `device`; owns an internal stream used by
 * helios_solve_re for graph capture. */
int helios_create(helios_ctx** ctx, int device);
int helios_destroy(helios_ctx* ctx);

/* Validate a batch, precompute its static geometry (Sect. 2.2.1: pressure
 * grid, sublayer column masses eq. 19, pressure-table indices), per-bin
 * constants (Planck prefactors, boundary spectra eqs. 20-22, two-stream
 * coefficients eqs. 8, 12-14), Gauss-Legendre weights (eqs. 31-32) and the
 * work list, and allocate the plan's workspace (warm-start fluxes, partial
 * sums, iteration state).  tables: host array of ntab descriptors whose
 * kappa pointers are device memory that must outlive the plan. */
int helios_plan_create(helios_ctx* ctx, const helios_batch_t* batch, const helios_ktable_t* tables, int ntab,
                       const helios_params_t* params, helios_plan** plan);
int helios_plan_destroy(helios_plan* plan);

/* Packed sizes of a plan: total layers, interfaces, points, bins; the number
 * of passes per temperature step (1 + n_scat if any omega0 > 0, else 1;
 * HELIOS_DIRECT with params.direct); bytes of workspace held; the sweep launches
 * per evaluation (one per group of atmospheres with the same lane chunk); whether
 * the bolometric sums join the temperature-step kernel (1) or run as their own
 * launch (0: an atmosphere with many work items); the sizes, in floats, of a
 * caller-owned warm-start buffer and of the per-bin flux output of
 * helios_flux_sweep. */
typedef struct {
    int64_t layers, interfaces, points, bins, cells;
    int passes;
    int64_t workspace_bytes;
    int sweep_launches;
    int fused_finalize;
    int64_t warm_floats;    /* floats of a warm-start buffer (helios_flux_sweep's Fup_warm) */
    int64_t spec_floats;    /* floats of the per-bin flux output (helios_flux_sweep's F_spec) */
} helios_plan_info_t;
int helios_plan_info(const helios_plan* plan, helios_plan_info_t* info);

/* Checkpoint and resume of an iteration (no counterpart in the paper).  Between steps a plan
 * keeps two things of its own: the upward fluxes of its last evaluation (the next warm start)
 * and that evaluation's point temperatures (from which the warm start is shifted to the new
 * temperatures).  With the caller's arrays (T_layer, mult, hist, nhist, status, iters) they are
 * the whole state of a radiative-equilibrium iteration: imported into this plan or into another
 * plan made from the same batch, tables and parameters, later steps continue the iteration bit
 * for bit.
 *   helios_plan_state_bytes: the size of a checkpoint
 *   helios_plan_state_export: copies this plan's state into buf (host or device memory,
 *     state_bytes long), queued on `stream`; EINVAL before the plan's first evaluation
 *   helios_plan_state_import: waits for `stream`, checks that buf holds a checkpoint of a plan
 *     of this shape (EINVAL otherwise), and queues the copies into the plan on `stream`; the next
 *     step with warm = 1 starts from it */
int helios_plan_state_bytes(const helios_plan* plan, int64_t* bytes);
int helios_plan_state_export(helios_plan* plan, void* buf, cudaStream_t stream);
int helios_plan_state_import(helios_plan* plan, const void* buf, cudaStream_t stream);

/* Measurement support (no counterpart in the paper).  helios_plan_set_timing
 * keeps a ring of `slots` CUDA event pairs (0 turns timing off; at most
 * 65536); while on, every helios_flux_sweep records a pair around its sweep
 * kernels on the launch stream (timing is suspended inside helios_solve_re's
 * graphs).  helios_plan_sweep_times waits for and returns the elapsed
 * milliseconds of the last min(max_n, slots, evaluations) sweeps, oldest first;
 * helios_plan_last_sweep_ms returns the last one. */
int helios_plan_set_timing(helios_plan* plan, int slots);
int helios_plan_sweep_times(helios_plan* plan, float* ms, int max_n, int* n_out);
int helios_plan_last_sweep_ms(helios_plan* plan, float* ms);

/* Opacity at every point, bin and Gauss point (Sect. 2.3): bilinear
 * interpolation of the k-table in (T, log10 P), T at interfaces the mean of
 * the adjacent centres (outer interfaces: the nearest centre).
 *   T_layer   device, double [layers]
 *   kappa_pts device, float, packed per atmosphere [2n+1][L][G]   (may be NULL)
 *   idx_pts   device, int32 [points][2] = (iP, iT)                (may be NULL)
 *   w_pts     device, double [points][2] = (wP, wT)               (may be NULL)
 * Indices and weights are computed in IEEE double without contraction and
 * match a plain C evaluation of the same formula bit for bit. */
int helios_interp_opacity(helios_plan* plan, const double* T_layer, float* kappa_pts, int32_t* idx_pts,
                          double* w_pts, cudaStream_t stream);

/* One flux evaluation at the temperatures T_layer (Sects. 2.1.3, 2.2.2,
 * 2.2.3, 2.3): opacities, sublayer optical depths (eq. 19), two-stream
 * transmission and coefficients (eqs. 8, 11-15; thin sublayers eq. 11,
 * pure scattering eq. 14), n_passes down/up passes with the boundary
 * conditions of eqs. 20 and 22, Gauss-point sum (eq. 31) and bin sum.
 *   T_layer  device, double [layers]
 *   n_passes >= 1, or 0 for the plan's default (1 + n_scat with scattering, or
 *            HELIOS_DIRECT when the plan's params.direct is set), or HELIOS_DIRECT
 *   warm     0: the coupled stream starts from zero (first temperature step);
 *            1: it starts from the upward fluxes of this plan's previous
 *               evaluation (later temperature steps, Sect. 2.2.3)
 *   Fup_warm device, float [warm_floats of helios_plan_info], 16-byte aligned, or
 *            NULL: the warm-start buffer (in/out; the upward fluxes of every
 *            column, as deviations from the local Planck flux, in the library's
 *            lane-interleaved layout).  NULL: the plan's own buffer.  Given, it
 *            replaces the plan's buffer for this call: with warm = 1 it must hold
 *            what an evaluation of this plan wrote into it, and the evaluation
 *            before this one must have been made at the temperatures that buffer
 *            was written at (the shift to the new temperatures uses the plan's
 *            record of the previous evaluation's point temperatures)
 *   Fup_bol, Fdn_bol  device, double [interfaces]: bolometric fluxes
 *   Fup_toa  device, float [bins]: emergent TOA spectrum per bin (may be NULL)
 *   F_spec   device, float [spec_floats of helios_plan_info] or NULL: a debug
 *            output of every bin's Gauss-point-summed fluxes at every point,
 *            packed per atmosphere as [L][2][2n+1] (upward at points 0..2n,
 *            then downward), atmosphere a starting at
 *            sum_{b<a} 2 L_b (2 n_b + 1)
 * Results are deterministic (fixed-order reductions). */
int helios_flux_sweep(helios_plan* plan, const double* T_layer, int n_passes, int warm, float* Fup_warm,
                      double* Fup_bol, double* Fdn_bol, float* Fup_toa, float* F_spec, cudaStream_t stream);

/* One temperature step (Sects. 2.2.3-2.2.4, eqs. 23-29) for every atmosphere
 * whose status is HELIOS_ATM_ACTIVE:
 *   dF_i = (Fup-Fdn)(i+1) - (Fup-Fdn)(i); if max_i |dF_i|/(sigma T_i^4) < tol
 *   the atmosphere becomes CONVERGED and T is left as is; otherwise
 *   dT_i = -mult_i f_pre t_rad dF_i/(rho_i c_p dz_i), T floored at T_floor, and
 *   the per-layer timestep multiplier follows the oscillation rule (six equal
 *   signs: x osc_up, capped at mult_max; any sign change among the last six:
 *   x osc_down).  All in double precision.
 *   Fup_bol, Fdn_bol device double [interfaces]; T_layer device double [layers] (in/out)
 *   mult  device double [layers] (in/out; start at 1)
 *   hist  device uint8 [layers] (in/out; bit 0 = newest sign, 1 = warming; start 0)
 *   nhist device uint8 [layers] (in/out; signs recorded so far, saturates at 6; start 0)
 *   status device int32 [A] (in/out), iters device int32 [A] (incremented; may be NULL)
 *   metric device double [A] (out: max |dF|/(sigma T^4); may be NULL) */
int helios_temp_update(helios_plan* plan, const double* Fup_bol, const double* Fdn_bol, double* T_layer,
                       double* mult, uint8_t* hist, uint8_t* nhist, int32_t* status, int32_t* iters,
                       double* metric, cudaStream_t stream);

/* One radiative-equilibrium iteration of every atmosphere (Sects. 2.2.3-2.2.4):
 * helios_flux_sweep with the plan's default passes followed by helios_temp_update,
 * as three launches (the bolometric sums, the metric and the temperature step are
 * one kernel per atmosphere).  Every atmosphere is evaluated whatever its status;
 * status[a] is recomputed from this step's metric (an atmosphere whose metric
 * meets eq. (29) keeps its temperatures) and iters[a] advances by one.
 *   T_layer, mult, hist, nhist, status, iters, metric: as helios_temp_update
 *   warm     as helios_flux_sweep
 *   Fup_bol, Fdn_bol  device, double [interfaces]: this step's bolometric fluxes
 *            (may be NULL: the plan's own buffers). */
int helios_re_step(helios_plan* plan, double* T_layer, int warm, double* mult, uint8_t* hist, uint8_t* nhist,
                   int32_t* status, int32_t* iters, double* metric, double* Fup_bol, double* Fdn_bol,
                   cudaStream_t stream);

/* helios_re_step for a caller whose temperatures live in host memory: copies
 * T_host into T_dev, makes one radiative-equilibrium iteration of every
 * atmosphere there, and copies the new temperatures back into T_host and the
 * statuses into status_host, all queued on `stream` (the host arrays hold the
 * step's result once the stream has reached this point; pinned host memory
 * makes the copies asynchronous).
 *   T_host      host double [layers] (in/out)
 *   T_dev       device double [layers], caller-owned scratch
 *   status_host host int32 [A] (out)
 *   the rest as helios_re_step (device arrays; the bolometric fluxes go to the
 *   plan's own buffers) */
int helios_re_step_host(helios_plan* plan, double* T_host, double* T_dev, int warm, double* mult, uint8_t* hist,
                        uint8_t* nhist, int32_t* status, int32_t* iters, double* metric, int32_t* status_host,
                        cudaStream_t stream);

/* The radiative-equilibrium iteration (Sect. 2.2.3): flux evaluation and
 * temperature step repeated, every atmosphere dropping out when it converges,
 * until none is active or max_iter evaluations were made.  The iteration runs
 * as CUDA graphs on the context's stream, ordered after the work already on
 * `stream`; the call returns when it is done.
 *   T_layer device double [layers]: start profile in, final profile out
 *   iters   device int32 [A] (out), status device int32 [A] (out)
 * Returns HELIOS_ENOCONV if any atmosphere ends NOT_CONVERGED or NONFINITE. */
int helios_solve_re(helios_plan* plan, double* T_layer, int32_t* iters, int32_t* status, cudaStream_t stream);

/* Learned initialiser (Sect. 2.2.3 starts the iteration from an arbitrary
 * profile; this network supplies a better one).  A multilayer perceptron
 * n_in -> hidden_layers x n_hidden (SiLU) -> n_out (linear), FP32 master
 * parameters; every matrix product rounds both operands to BF16 and accumulates
 * in FP32 on the 5th-generation tensor cores (tcgen05 MMAs with the accumulator
 * in tensor memory, 128 x 64 output tiles; the weight operand reaches shared memory as
 * pre-tiled BF16 by bulk asynchronous copies).  Parameter layout (device, float): for each layer
 * l, W_l [in][out] row-major then b_l [out].  Initial weights are uniform in
 * +-1/sqrt(fan_in) from `seed`.  Batches hold up to max_batch rows.
 *   helios_mlp_forward: y[B][n_out] = net(x[B][n_in]) (device arrays)
 *   helios_mlp_grad: gradient of the mean squared error mean((net(x) - target)^2)
 *     into the internal gradient buffer (readable through helios_mlp_params);
 *     loss (device float, may be NULL)
 *   helios_mlp_adam: one Adam step (bias-corrected) on the parameters
 *   helios_mlp_train_step: grad + Adam(lr, 0.9, 0.999, 1e-8)
 * All calls are asynchronous on `stream`; reductions have a fixed order. */
typedef struct helios_mlp helios_mlp;
int helios_mlp_create(helios_ctx* ctx, int n_in, int n_hidden, int hidden_layers, int n_out,
                      unsigned long long seed, int max_batch, helios_mlp** mlp);
int helios_mlp_destroy(helios_mlp* mlp);
int helios_mlp_params(helios_mlp* mlp, float** params, float** grads, long long* count);
/* The matrix products read the weights from a BF16 copy laid out in the tensor cores' shared-memory
 * tile order (both orientations, built from the FP32 parameters before the first product and kept
 * current by every helios_mlp_adam).  A caller that writes the parameters through the pointer of
 * helios_mlp_params declares it here, so that the copy is rebuilt before the next product (on the
 * stream of that product).  No counterpart in the paper. */
int helios_mlp_params_changed(helios_mlp* mlp);
/* Synchronous: *flag = 1 if a matrix product of this network gave up waiting for its tensor-core
 * operations (a bounded wait that expired; its results are then invalid), else 0. */
int helios_mlp_error(helios_mlp* mlp, int* flag);
int helios_mlp_forward(helios_mlp* mlp, const float* x, float* y, int B, cudaStream_t stream);
int helios_mlp_grad(helios_mlp* mlp, const float* x, const float* target, int B, float* loss, cudaStream_t stream);
int helios_mlp_adam(helios_mlp* mlp, float lr, float beta1, float beta2, float eps, cudaStream_t stream);
int helios_mlp_train_step(helios_mlp* mlp, const float* x, const float* target, int B, float lr, float* loss,
                          cudaStream_t stream);

/* Training-data preparation of the learned initialiser: per column j of x
 * (device float [B][n]) the mean and the population standard deviation plus
 * eps, accumulated in double in a fixed order (helios_column_stats: mu, sd
 * device float [n], out); and xs = (x - mu)/sd column-wise in IEEE float32
 * (helios_standardize: xs device float [B][n], may alias x).  Asynchronous. */
int helios_column_stats(const float* x, int B, int n, double eps, float* mu, float* sd, cudaStream_t stream);
int helios_standardize(const float* x, const float* mu, const float* sd, int B, int n, float* xs, cudaStream_t stream);

/* Start profiles of a plan's atmospheres from the learned initialiser (the
 * iteration of Sect. 2.2.3 may start from any profile; this one is closer to
 * equilibrium).  Per atmosphere a: its features feats[a] (device float
 * [A][n_in], raw values) are standardised, (f - x_mu)/x_sd in IEEE float32;
 * the network maps them to n_out standardised temperatures at evenly spaced
 * normalised log-P positions k/(n_out - 1), bottom first; these are
 * de-standardised, t = y * y_sd + y_mu, and interpolated linearly in log P to
 * the atmosphere's n layer centres (evenly spaced in log P: layer i at
 * i/(n - 1)), in double precision.  A profile with a non-finite temperature or
 * one outside (T_min, T_max) is replaced by the atmosphere's T_fallback.
 *   x_mu, x_sd device float [n_in]; y_mu, y_sd device float [n_out]
 *   T_fallback, T_layer device double [layers] (T_layer: out)
 *   used device int32 [A] (out: 1 where the network's profile was kept; may be NULL)
 * Processes max_batch atmospheres per network pass; asynchronous on `stream`. */
int helios_mlp_initial_profiles(helios_mlp* mlp, const helios_plan* plan, const float* feats, const float* x_mu,
                                const float* x_sd, const float* y_mu, const float* y_sd, const double* T_fallback,
                                double T_min, double T_max, double* T_layer, int32_t* used, cudaStream_t stream);

/* Autotuner (measurement support; the paper has no counterpart): picks the work
 * item size (bins_per_item) and launch mode (persistent) for a batch by timing
 * one flux evaluation of a calibration subset (up to 128 atmospheres spread over
 * the batch) for each candidate, and returns `base` with the fastest choice in
 * `tuned`.  The choice is cached in the JSON file cache_path (may be NULL) under a
 * key made of the device name and the batch's shape bucket (log2 of A, mean
 * layers, mean bins, G, scattering or not); a cached key is returned without
 * timing.  Allocates and frees its own temporary plans and buffers; synchronous. */
int helios_autotune(helios_ctx* ctx, const helios_batch_t* batch, const helios_ktable_t* tables, int ntab,
                    const helios_params_t* base, const char* cache_path, helios_params_t* tuned);

/* Measured FP32-FMA throughput (TFLOP/s, an FMA counted as 2) and MUFU ex2
 * throughput (T op/s) of the context's device, from independent dependency chains
 * filling every SM (the paper has no counterpart): the denominators of the sweep's
 * FP32-issue and SFU roofline terms.  Synchronous; allocates and frees a small buffer. */
int helios_measure_peaks(helios_ctx* ctx, double* fp32_tflops, double* sfu_tops);

/* y[i] = 1/x[i], i < n, by the device reciprocal of the two-stream coefficients (the
 * hardware's approximate reciprocal refined by one Newton-Raphson step): a check of that
 * routine against correctly rounded quotients (no counterpart in the paper).  x, y: device
 * float arrays of n >= 0 elements (x normal and positive for the stated accuracy); async on
 * `stream`.  HELIOS_EINVAL for a null array with n > 0 or n < 0. */
int helios_device_recip(const float* x, float* y, int n, cudaStream_t stream);

/* Allocation-free flux evaluation (the paper has no counterpart; it exists for
 * callers that cannot allocate device memory -- code running under a framework
 * that owns the device's memory pool, or in a region where cudaMalloc is not
 * allowed).  Same computation as helios_flux_sweep from a cold start (the coupled
 * stream starts from zero) for ONE atmosphere (batch->A == 1, host arrays as in
 * helios_batch_t), without a plan: the call performs no cudaMalloc, cudaFree or
 * other allocation, on the device or the host.  Its working memory is one 64 MiB
 * array held, as a static device object of the library, by every GPU that runs
 * the library's code until the process exits.
 *   table   host descriptor; kappa device pointer (as in helios_ktable_t)
 *   T_layer device double [n]; Fup_bol, Fdn_bol device double [n+1];
 *   Fup_toa device float [L] or NULL; n_passes as in helios_flux_sweep.
 * The first call on a device looks up the array's device address (with that
 * device current).  The call stages its inputs through static host arrays with
 * pageable copies, so it cannot be captured in a CUDA graph: on a stream that is
 * capturing it returns HELIOS_EINVAL without queueing work.  Atmospheres beyond
 * n_layers 239, n_bins 8192 or G 20 are rejected with HELIOS_EINVAL before any GPU
 * work; every atmosphere within those limits fits (no warm start is kept).  All
 * calls share the array and each call rewrites it entirely before reading it;
 * calls whose GPU work overlaps (different streams or host threads without
 * ordering) race on it.  The host set-up is the plan's own; results equal
 * helios_flux_sweep with warm = 0 up to the order of the final FP64 sums. */
int helios_flux_sweep_noalloc(const helios_batch_t* batch, const helios_ktable_t* table,
                              const helios_params_t* params, const double* T_layer, int n_passes,
                              double* Fup_bol, double* Fdn_bol, float* Fup_toa, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif
