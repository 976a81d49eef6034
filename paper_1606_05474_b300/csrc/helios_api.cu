// C ABI of the radiative-equilibrium hot path: validation, plan set-up (static
// geometry and per-bin constants in double precision on the host), kernel
// launches and the CUDA-graph radiative-equilibrium loop.  See include/helios.h.
#include "helios.h"
#include "helios_kernels.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "helios_setup.h"

#include <nvtx3/nvToolsExt.h>

// a named range on a profiler's timeline around each call of the boundary (nothing is recorded
// when no tool is attached)
namespace {
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
};
}  // namespace

using namespace helios_dev;
using namespace helios_setup;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(HELIOS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr int kMaxG = 20;           // 32 G threads per block <= 640
constexpr int kMaxM = 15;           // 2n+1 <= 32*15  ->  n <= 239
constexpr int kMaxN = (32 * kMaxM - 1) / 2;

// sublayer slots per lane of a column spread over cl lanes (odd: conflict-free smem rows)
int lane_chunk(int n, int cl = 32)
{
    int m = (2 * n + 1 + cl - 1) / cl;
    if (!(m & 1)) ++m;
    return m;
}


template <typename T>
int dev_alloc(T** p, size_t count, size_t& total)
{
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(HELIOS_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    total += bytes;
    return HELIOS_OK;
}

template <typename T>
int upload(T* dst, const std::vector<T>& src)
{
    if (src.empty()) return HELIOS_OK;
    CUDA_TRY(cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return HELIOS_OK;
}

size_t sweep_smem(int M, int G, int cl = 32) { return sweep_smem_bytes(M, G, cl); }

// atmospheres of at most this many work items have their bolometric sums done by the
// per-atmosphere temperature-step block (post_kernel); wider ones by finalize_kernel
constexpr int kFuseFinalizeItems = 64;

// 16-lane columns (two per warp), 320-thread blocks: three per SM (64 registers, a few spilled)
// up to lane chunk 11, two (96 registers) beyond.  Measured on the full-size bins: three blocks
// are 5-14 % faster than two up to chunk 11; four at chunks 5-7 were slower again
template <int M> constexpr int minb16() { return M <= 11 ? 3 : 2; }

template <int M, bool DIRECT, int CL = 32>
int sweep_occupancy_MD(int threads, size_t smem)
{
    int nb = 0;
    auto k = [] {
        if constexpr (CL == 16) return sweep_kernel<M, minb16<M>(), false, 16>;
        else return sweep_kernel<M, sweep_minb<M, DIRECT>(), DIRECT>;
    }();
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem) != cudaSuccess)
        return 0;
    return nb;
}

template <int M>
int sweep_occupancy_M(int threads, size_t smem, bool direct)
{
    return direct ? sweep_occupancy_MD<M, true>(threads, smem) : sweep_occupancy_MD<M, false>(threads, smem);
}

// lane chunks of 16-lane columns: 24 to 119 layers (chunk 15 is the largest that two 320-thread
// blocks per SM hold in registers with little spilling)
constexpr bool cl16_chunk(int M) { return M >= 5 && M <= 15; }

// lanes per column of an atmosphere of n layers for the request 0 (automatic), 16 or 32; 0 if
// 16 was requested outside its range.  Measured on the full-size bins (3000 x 20 g, 5 passes),
// 16 lanes are 7-25 % faster than 32 everywhere in that range
int column_lanes(int n, int request)
{
    if (request == 32) return 32;
    return cl16_chunk(lane_chunk(n, 16)) ? 16 : (request == 16 ? 0 : 32);
}

// group key of the iterated sweep's launches: (lanes per column, lane chunk)
constexpr int kGroups = 2 * (kMaxM + 1);
constexpr int group_key(int cl, int M) { return (cl == 16 ? kMaxM + 1 : 0) + M; }

// resident sweep blocks per SM for lane chunk M, block size, dynamic shared memory, mode and
// lanes per column (0 on error)
int sweep_occupancy(int M, int threads, size_t smem, bool direct = false, int cl = 32)
{
    if (cl == 16) {
        switch (M) {
            case 5: return sweep_occupancy_MD<5, false, 16>(threads, smem);
            case 7: return sweep_occupancy_MD<7, false, 16>(threads, smem);
            case 9: return sweep_occupancy_MD<9, false, 16>(threads, smem);
            case 11: return sweep_occupancy_MD<11, false, 16>(threads, smem);
            case 13: return sweep_occupancy_MD<13, false, 16>(threads, smem);
            case 15: return sweep_occupancy_MD<15, false, 16>(threads, smem);
            default: return 0;
        }
    }
    switch (M) {
        case 1: return sweep_occupancy_M<1>(threads, smem, direct);
        case 3: return sweep_occupancy_M<3>(threads, smem, direct);
        case 5: return sweep_occupancy_M<5>(threads, smem, direct);
        case 7: return sweep_occupancy_M<7>(threads, smem, direct);
        case 9: return sweep_occupancy_M<9>(threads, smem, direct);
        case 11: return sweep_occupancy_M<11>(threads, smem, direct);
        case 13: return sweep_occupancy_M<13>(threads, smem, direct);
        case 15: return sweep_occupancy_M<15>(threads, smem, direct);
        default: return 0;
    }
}

}  // namespace

__attribute__((visibility("hidden"))) void helios_set_error_text(const char* msg) { g_err = msg; }

struct helios_ctx {
    int device;
    cudaStream_t stream;
    cudaEvent_t ev_in, ev_out;
    int* h_active;    // pinned
};

struct MGroup {
    int M;            // lane chunk of the iterated sweep
    int cl;           // its lanes per column (16 or 32)
    int threads;      // its block size
    int M_direct;     // lane chunk of the exact column solve (32 lanes per column)
    int count;
    int* order;       // device
    int* counter;     // device work counters of persistent launches: [items pulled, blocks done]
    int grid;         // persistent grid: resident blocks on all SMs
    int grid_direct;  // the same for the direct column solve
    cudaStream_t stream;   // the group's own stream (several groups overlap)
    cudaEvent_t join;
};

struct helios_plan {
    helios_ctx* ctx;
    helios_params_t prm;
    int A, G, TB, passes, max_n;
    int64_t layers, interfaces, points, subs, bins, items, cells;
    int64_t ws_bytes;
    int2* lay_nl;           // device [A]: (layers, first layer) of each atmosphere
    int64_t warm_floats;    // floats of the warm-start block (all atmospheres)
    int64_t spec_floats;    // floats of the optional per-bin flux output [bins][2][points]
    std::vector<AtmDesc> atms_h;
    std::vector<MGroup> groups;
    PlanDev dev;
    std::vector<void*> allocs;
    // solve state
    double *Fup, *Fdn, *mult;
    uint8_t *hist, *nhist;
    int* n_active;
    bool warm_ready;
    int64_t state_hdr[4];   // header of an exported checkpoint (host memory of a pending copy)
    cudaGraphExec_t graph;
    const void* graph_key[3];
    int graph_chunk;
    int graph_device_loop;
    int max_items;      // work items of the widest atmosphere
    int* chunks_left;   // device budget of WHILE-node iterations (device_loop)
    cudaEvent_t fork;
    int* counters;
    // optional timing of the sweep kernels: a ring of event pairs on the launch stream
    int timing;
    std::vector<cudaEvent_t> ev_ring;
    int64_t n_timed;
    cudaEvent_t ev_sweep0, ev_sweep1;   // the pair used by the current evaluation
};

__attribute__((visibility("hidden"))) int helios_ctx_device(const helios_ctx* c) { return c->device; }

// per atmosphere (layers, offset of its first layer) on the device, for the learned initialiser
__attribute__((visibility("hidden"))) const int2* helios_plan_layers_dev(const helios_plan* p, int* A)
{
    *A = p->A;
    return p->lay_nl;
}

extern "C" {

void helios_default_params(helios_params_t* p)
{
    if (!p) return;
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
    p->n_scat = 4;
    p->max_iter = 20000;
    p->grey_mode = 0;
    p->printed_gradient = 0;
    p->bins_per_item = 0;
    p->check_every = 0;
    p->persistent = 1;
    p->iso_layers = 0;
    p->device_loop = 1;
    p->direct = 0;
    p->rayleigh = 0;
    p->col_lanes = 0;
    p->tabulate = 0;
}

int helios_version(void) { return HELIOS_VERSION; }

const char* helios_last_error(void) { return g_err.c_str(); }

int helios_create(helios_ctx** out, int device)
{
    if (!out) return fail(HELIOS_EINVAL, "helios_create: null output pointer");
    *out = nullptr;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(HELIOS_EINVAL, "helios_create: device %d of %d", device, ndev);
    CUDA_TRY(cudaSetDevice(device));
    helios_ctx* c = new helios_ctx();
    c->device = device;
    CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    CUDA_TRY(cudaMallocHost((void**)&c->h_active, sizeof(int)));
    *out = c;
    return HELIOS_OK;
}

int helios_destroy(helios_ctx* c)
{
    if (!c) return HELIOS_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->stream);
    cudaEventDestroy(c->ev_in);
    cudaEventDestroy(c->ev_out);
    cudaFreeHost(c->h_active);
    delete c;
    return HELIOS_OK;
}

int helios_plan_destroy(helios_plan* p)
{
    if (!p) return HELIOS_OK;
    cudaSetDevice(p->ctx->device);
    cudaDeviceSynchronize();
    if (p->graph) cudaGraphExecDestroy(p->graph);
    for (MGroup& g : p->groups) {
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.join) cudaEventDestroy(g.join);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    for (cudaEvent_t e : p->ev_ring) cudaEventDestroy(e);
    for (void* a : p->allocs) cudaFree(a);
    delete p;
    return HELIOS_OK;
}

int helios_plan_create(helios_ctx* ctx, const helios_batch_t* b, const helios_ktable_t* tabs, int ntab,
                       const helios_params_t* prm, helios_plan** out)
{
    CallRange range_("helios_plan_create");
    if (!out) return fail(HELIOS_EINVAL, "helios_plan_create: null output pointer");
    *out = nullptr;
    if (!ctx || !b || !tabs || !prm) return fail(HELIOS_EINVAL, "helios_plan_create: null argument");
    if (b->A < 1) return fail(HELIOS_EINVAL, "batch has %d atmospheres", b->A);
    if (ntab < 1) return fail(HELIOS_EINVAL, "no k-table given");
    if (!b->n_layers || !b->n_bins || !b->table_id || !b->P_top_bar || !b->P_bot_bar || !b->grav || !b->T_irr ||
        !b->T_int || !b->T_star || !b->nu_edges || !b->omega0 || !b->g0)
        return fail(HELIOS_EINVAL, "batch has a null array");
    if (!(prm->D > 0.0) || !(prm->dtau_iso >= 0.0) || !(prm->w0_pure >= 0.0) || !(prm->tol > 0.0) ||
        prm->n_scat < 0 || prm->max_iter < 1 || !(prm->osc_down > 0.0) || !(prm->osc_up > 0.0) ||
        !(prm->mult_max > 0.0) || !(prm->T_floor > 0.0) || prm->bins_per_item < 0 || prm->check_every < 0 ||
        prm->persistent < 0 || prm->persistent > 1 || prm->iso_layers < 0 || prm->iso_layers > 1 ||
        prm->device_loop < 0 || prm->device_loop > 1 || prm->direct < 0 || prm->direct > 1 ||
        prm->rayleigh < 0 || prm->rayleigh > 1 || (prm->rayleigh && prm->grey_mode) ||
        (prm->col_lanes != 0 && prm->col_lanes != 16 && prm->col_lanes != 32) || prm->tabulate < 0 ||
        prm->tabulate > 1)
        return fail(HELIOS_EINVAL, "invalid parameter set");
    if (prm->tabulate && (prm->iso_layers || prm->direct || prm->rayleigh || prm->grey_mode))
        return fail(HELIOS_EINVAL, "tabulated functions: not with iso_layers, direct, rayleigh or grey_mode");
    const int G = tabs[0].G;
    if (G < 1 || G > kMaxG) return fail(HELIOS_EINVAL, "G = %d outside [1, %d]", G, kMaxG);
    for (int t = 0; t < ntab; ++t) {
        const helios_ktable_t& k = tabs[t];
        if (k.G != G) return fail(HELIOS_EINVAL, "table %d has G = %d, table 0 has %d", t, k.G, G);
        if (k.nP < 1 || k.nT < 1 || k.L < 1) return fail(HELIOS_EINVAL, "table %d has an empty axis", t);
        if ((k.nP > 1 && !(k.dlog10P > 0.0)) || (k.nT > 1 && !(k.dT > 0.0)))
            return fail(HELIOS_EINVAL, "table %d has a non-increasing axis", t);
        if (!k.kappa || ((uintptr_t)k.kappa & 15)) return fail(HELIOS_EINVAL, "table %d: kappa null or not 16-byte aligned", t);
    }
    if (prm->grey_mode) {
        for (int a = 0; a < b->A; ++a)
            if (b->n_bins[a] != 2) return fail(HELIOS_EINVAL, "grey mode needs exactly 2 bins (atmosphere %d)", a);
    }
    CUDA_TRY(cudaSetDevice(ctx->device));

    helios_plan* P = new helios_plan();
    P->ctx = ctx;
    P->prm = *prm;
    P->A = b->A;
    P->G = G;
    P->graph = nullptr;
    P->warm_ready = false;

    // ---- per-atmosphere layout
    const int A = b->A;
    std::vector<AtmDesc> ad(A);
    int64_t lay = 0, ifc = 0, pts = 0, sub = 0, bins = 0, nu_off = 0;
    for (int a = 0; a < A; ++a) {
        const int n = b->n_layers[a], L = b->n_bins[a], t = b->table_id[a];
        if (n < 2 || n > kMaxN) { delete P; return fail(HELIOS_EINVAL, "atmosphere %d: n_layers = %d outside [2, %d]", a, n, kMaxN); }
        if (L < 1) { delete P; return fail(HELIOS_EINVAL, "atmosphere %d: n_bins = %d", a, L); }
        if (t < 0 || t >= ntab) { delete P; return fail(HELIOS_EINVAL, "atmosphere %d: table_id %d", a, t); }
        if (L > tabs[t].L) { delete P; return fail(HELIOS_EINVAL, "atmosphere %d: %d bins > table %d's %d", a, L, t, tabs[t].L); }
        if (!(b->P_top_bar[a] > 0.0) || !(b->P_bot_bar[a] > b->P_top_bar[a]) || !(b->grav[a] > 0.0) ||
            !(b->T_irr[a] >= 0.0) || !(b->T_int[a] >= 0.0) || !(b->T_star[a] > 0.0) ||
            !std::isfinite(b->P_bot_bar[a]) || !std::isfinite(b->T_irr[a]) || !std::isfinite(b->T_int[a])) {
            delete P;
            return fail(HELIOS_EINVAL, "atmosphere %d: invalid pressure range, gravity or temperatures", a);
        }
        for (int l = 0; l <= L; ++l) {
            const double v = b->nu_edges[nu_off + l];
            if (!(v > 0.0) || !std::isfinite(v) || (l > 0 && !(v > b->nu_edges[nu_off + l - 1]))) {
                delete P;
                return fail(HELIOS_EINVAL, "atmosphere %d: bin edges must be positive and increasing", a);
            }
        }
        for (int l = 0; l < L; ++l) {
            const float w0 = b->omega0[bins + l], g0 = b->g0[bins + l];
            if (!(w0 >= 0.0f && w0 <= 1.0f) || !(g0 >= -1.0f && g0 <= 1.0f) ||
                (!(1.0 - (double)w0 < prm->w0_pure) && !(w0 < 1.0f))) {
                delete P;
                return fail(HELIOS_EINVAL, "atmosphere %d bin %d: omega0 %g / g0 %g invalid", a, l, w0, g0);
            }
        }
        AtmDesc& d = ad[a];
        std::memset(&d, 0, sizeof d);
        d.cl = column_lanes(n, prm->col_lanes);
        if (!d.cl) {
            delete P;
            return fail(HELIOS_EINVAL, "atmosphere %d: n_layers = %d outside [24, 119] for 16-lane columns", a, n);
        }
        d.n = n; d.L = L; d.M = lane_chunk(n, d.cl); d.tab = t;
        if (b->species_off) {
            const int s0 = b->species_off[a], s1 = b->species_off[a + 1];
            if (!b->species_table || !b->species_weight || s1 < s0 || s1 - s0 > 16 || s0 < 0) {
                delete P;
                return fail(HELIOS_EINVAL, "atmosphere %d: invalid species range", a);
            }
            for (int j = s0; j < s1; ++j) {
                const int tj = b->species_table[j];
                const double wj = b->species_weight[j];
                if (tj < 0 || tj >= ntab || !(wj >= 0.0) || !std::isfinite(wj)) {
                    delete P;
                    return fail(HELIOS_EINVAL, "atmosphere %d: species %d table %d weight %g invalid", a, j, tj, wj);
                }
                const helios_ktable_t &k0 = tabs[t], &kj = tabs[tj];
                if (kj.nP != k0.nP || kj.nT != k0.nT || kj.L != k0.L || kj.G != k0.G || kj.log10P0 != k0.log10P0 ||
                    kj.dlog10P != k0.dlog10P || kj.T0 != k0.T0 || kj.dT != k0.dT) {
                    delete P;
                    return fail(HELIOS_EINVAL, "atmosphere %d: species table %d does not share table %d's grid", a, tj, t);
                }
            }
            d.n_spec = s1 - s0;
            d.spec_off = s0;
        }
        d.lay_off = (int)lay; d.if_off = (int)ifc; d.pt_off = (int)pts; d.sub_off = (int)sub; d.bin_off = (int)bins;
        lay += n; ifc += n + 1; pts += 2 * n + 1; sub += 2 * n; bins += L; nu_off += L + 1;
    }
    if (pts > INT32_MAX / 2 || bins > INT32_MAX / 2) { delete P; return fail(HELIOS_EINVAL, "batch too large"); }
    P->max_n = 0;
    for (int a = 0; a < A; ++a) P->max_n = std::max(P->max_n, ad[a].n);
    P->layers = lay; P->interfaces = ifc; P->points = pts; P->subs = sub; P->bins = bins;
    int64_t cells = 0;
    for (int a = 0; a < A; ++a) cells += (int64_t)ad[a].n * ad[a].L * G;
    P->cells = cells;

    // ---- work items: tiles of TB bins
    // bins per work item: one resident wave of blocks (at the sweep occupancy of the widest
    // atmosphere) for a single atmosphere, capped for long batches so the tail stays short.
    // Block (iterated passes): one warp per two Gauss points
    const int threads = sweep_block_threads(G, false);
    int amax = 0;
    for (int a = 0; a < A; ++a)
        if (ad[a].n > ad[amax].n) amax = a;
    int TB = prm->bins_per_item;
    if (TB <= 0) {
        int nsm = 148;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
        const int cm = ad[amax].cl, mm = ad[amax].M;
        const int per_sm = std::max(1, sweep_occupancy(mm, threads, sweep_smem(mm, G, cm), false, cm));
        const int64_t slots = (int64_t)nsm * per_sm;
        TB = (int)std::max<int64_t>(1, std::min<int64_t>(32, (bins + slots - 1) / slots));
        // a batch of at least four waves of 8-bin items takes items of 8 bins: once most
        // atmospheres of a radiative-equilibrium solve have converged, an iteration of the rest
        // lasts as long as one item's bins one after the other (measured on 512 atmospheres of 300
        // bins: 20% less solve time than 32-bin items, 2% more time per step with all active)
        if (bins >= 4 * slots * 8) TB = std::min(TB, 8);
    }
    P->TB = TB;
    std::vector<int2> items;
    int64_t part = 0, warm = 0, fspec = 0;
    for (int a = 0; a < A; ++a) {
        AtmDesc& d = ad[a];
        d.n_items = (d.L + TB - 1) / TB;
        P->max_items = std::max(P->max_items, d.n_items);
        d.item_off = (int)items.size();
        for (int t = 0; t < d.n_items; ++t) items.push_back(make_int2(a, t));
        d.part_off = part;
        part += (int64_t)d.n_items * 3 * (d.n + 1);
        d.warm_off = warm;
        warm += (int64_t)d.L * G * d.cl * d.M;
        d.fspec_off = fspec;
        fspec += (int64_t)d.L * 2 * (2 * d.n + 1);
    }
    P->warm_floats = warm;
    P->spec_floats = fspec;
    P->items = (int64_t)items.size();
    // launch order per group (lanes per column, lane chunk), most expensive items first
    std::vector<std::vector<int>> byM(kGroups);
    for (int i = 0; i < (int)items.size(); ++i) byM[group_key(ad[items[i].x].cl, ad[items[i].x].M)].push_back(i);
    for (int key = 0; key < kGroups; ++key) {
        auto& v = byM[key];
        std::stable_sort(v.begin(), v.end(), [&](int x, int y) {
            const AtmDesc& a = ad[items[x].x];
            const AtmDesc& c = ad[items[y].x];
            int ca = a.n * std::min(TB, a.L - items[x].y * TB), cb = c.n * std::min(TB, c.L - items[y].y * TB);
            return ca > cb;
        });
    }

    // ---- static geometry (Sect. 2.2.1, eq. 19) and pressure-table coordinates
    std::vector<int> iP(pts), lay_atm(lay);
    std::vector<double> wP(pts), lnr(lay);
    std::vector<float> dm(sub);
    for (int a = 0; a < A; ++a) {
        const AtmDesc& d = ad[a];
        std::vector<double> Pp(2 * d.n + 1);
        layer_geometry(d.n, b->P_bot_bar[a], b->P_top_bar[a], b->grav[a], prm->iso_layers, tabs[d.tab], Pp.data(),
                       &iP[d.pt_off], &wP[d.pt_off], &dm[d.sub_off], &lnr[d.lay_off]);
        for (int i = 0; i < d.n; ++i) lay_atm[d.lay_off + i] = a;
    }

    // ---- per-bin constants (eqs. 8, 12-14, 20-22), double precision then rounded
    const double D = prm->D, eps = 1.0 / D;
    std::vector<BinConst> bc(bins);
    // Sect. 2.6 tables: 2 pi eps B of every bin at the 10 K nodes (the same quantity the sweep
    // otherwise forms as E / (e^x - 1)), and 1 - e^-x at the 0.1-dex nodes of x
    std::vector<float> btab, utab;
    if (prm->tabulate) {
        if (bins * (int64_t)kTabNT > ((int64_t)1 << 30)) {
            delete P;
            return fail(HELIOS_EINVAL, "tabulated Planck functions: %lld bins are too many", (long long)bins);
        }
        btab.resize((size_t)bins * kTabNT);
        utab.resize(2 * kTabNX);
        for (int i = 0; i < kTabNX; ++i) {
            const double x = std::pow(10.0, (double)kTabX0 + 0.1 * i);
            utab[i] = (float)x;
            utab[kTabNX + i] = (float)(-std::expm1(-x));
        }
    }
    bool any_scat = false;
    nu_off = 0;
    for (int a = 0; a < A; ++a) {
        const AtmDesc& d = ad[a];
        const double* e = b->nu_edges + nu_off;
        any_scat |= bin_constants(e, b->omega0 + d.bin_off, b->g0 + d.bin_off, d.L, b->T_irr[a], b->T_int[a],
                                  b->T_star[a], *prm, &bc[d.bin_off]);
        if (prm->tabulate)
            for (int l = 0; l < d.L; ++l)
                for (int j = 0; j < kTabNT; ++j)
                    btab[(size_t)(d.bin_off + l) * kTabNT + j] =
                        (float)(2.0 * kPi * eps * planck_bin(e[l], e[l + 1], j * (double)kTabDT));
        nu_off += d.L + 1;
    }
    P->passes = prm->direct ? HELIOS_DIRECT : (any_scat ? 1 + prm->n_scat : 1);

    // ---- Gauss weights on [0, 1]
    std::vector<float> gw(G);
    gauss_weights01(G, gw.data());

    std::vector<TabDesc> td(ntab);
    for (int t = 0; t < ntab; ++t) {
        td[t].kappa = tabs[t].kappa;
        td[t].nP = tabs[t].nP; td[t].nT = tabs[t].nT; td[t].L = tabs[t].L; td[t].G = tabs[t].G;
        td[t].log10P0 = tabs[t].log10P0; td[t].dlog10P = tabs[t].dlog10P;
        td[t].T0 = tabs[t].T0; td[t].dT = tabs[t].dT;
        td[t].rowL = tabs[t].L * tabs[t].G;
        td[t].offP = tabs[t].nP > 1 ? tabs[t].nT * td[t].rowL : 0;
        td[t].offT = tabs[t].nT > 1 ? td[t].rowL : 0;
        if ((int64_t)tabs[t].nP * tabs[t].nT * tabs[t].L * tabs[t].G >= ((int64_t)1 << 31)) {
            delete P;
            return fail(HELIOS_EINVAL, "table %d has 2^31 or more entries", t);
        }
    }

    // ---- device workspace
    size_t tot = 0;
    int rc = HELIOS_OK;
    PlanDev& dv = P->dev;
    std::memset(&dv, 0, sizeof dv);
    AtmDesc* d_atm; TabDesc* d_tab; BinConst* d_bc; int2* d_items; int* d_order; float* d_gw;
    int* d_iP; double* d_wP; float* d_dm; double* d_lnr; int* d_lay_atm; int* d_spec_tab; float* d_spec_w;
    std::vector<int> spec_tab;
    std::vector<float> spec_w;
    if (b->species_off) {
        for (int j = 0; j < b->species_off[A]; ++j) {
            spec_tab.push_back(b->species_table[j]);
            spec_w.push_back((float)b->species_weight[j]);
        }
    }
#define ALLOC(ptr, cnt)                                              \
    do {                                                             \
        if ((rc = dev_alloc(&ptr, (cnt), tot)) != HELIOS_OK) {       \
            helios_plan_destroy(P);                                  \
            return rc;                                               \
        }                                                            \
        P->allocs.push_back((void*)ptr);                             \
    } while (0)
    ALLOC(d_atm, A); ALLOC(d_tab, ntab); ALLOC(d_bc, bins); ALLOC(d_items, items.size());
    ALLOC(d_order, items.size()); ALLOC(d_gw, G); ALLOC(d_iP, pts); ALLOC(d_wP, pts); ALLOC(d_dm, sub);
    ALLOC(d_lnr, lay); ALLOC(d_lay_atm, lay); ALLOC(d_spec_tab, spec_tab.size()); ALLOC(d_spec_w, spec_w.size());
    ALLOC(dv.row, pts); ALLOC(dv.wq, pts);
    ALLOC(dv.Tpt, pts); ALLOC(dv.iT, pts); ALLOC(dv.wT, pts); ALLOC(dv.invT, pts); ALLOC(dv.Tf, pts);
    ALLOC(dv.invT_old, pts); ALLOC(dv.dinv_step, pts); ALLOC(dv.dT_step, pts);
    ALLOC(dv.dinv_sub, sub); ALLOC(dv.dT_sub, sub);
    ALLOC(dv.part, part); ALLOC(dv.warm, warm);
    ALLOC(P->Fup, ifc); ALLOC(P->Fdn, ifc); ALLOC(P->mult, lay); ALLOC(P->hist, lay); ALLOC(P->nhist, lay);
    ALLOC(P->n_active, 1); ALLOC(P->chunks_left, 1);
    ALLOC(P->counters, 2 * kGroups);
    ALLOC(P->lay_nl, A);
    float *d_btab = nullptr, *d_utab = nullptr;
    if (prm->tabulate) {
        ALLOC(d_btab, btab.size());
        ALLOC(d_utab, utab.size());
    }
#undef ALLOC
    std::vector<int> order;
    int nsm_all = 148;
    cudaDeviceGetAttribute(&nsm_all, cudaDevAttrMultiProcessorCount, ctx->device);
    for (int key = 0; key < kGroups; ++key) {
        if (byM[key].empty()) continue;
        MGroup gr;
        std::memset(&gr, 0, sizeof gr);
        gr.cl = key > kMaxM ? 16 : 32;
        gr.M = key - (gr.cl == 16 ? kMaxM + 1 : 0);
        gr.threads = threads;
        // the exact solve runs 32 lanes per column: a chunk covering the group's longest column
        gr.M_direct = gr.cl == 32 ? gr.M : lane_chunk((gr.cl * gr.M - 1) / 2, 32);
        gr.count = (int)byM[key].size();
        gr.order = d_order + order.size();
        gr.counter = P->counters + 2 * key;     // [work items pulled, blocks finished]
        gr.grid = std::min(gr.count, nsm_all * std::max(1, sweep_occupancy(gr.M, gr.threads,
                                                                          sweep_smem(gr.M, G, gr.cl), false, gr.cl)));
        gr.grid_direct = std::min(gr.count, nsm_all * std::max(1, sweep_occupancy(gr.M_direct, 32 * G,
                                                                                 sweep_smem(gr.M_direct, G), true)));
        order.insert(order.end(), byM[key].begin(), byM[key].end());
        P->groups.push_back(gr);
    }
    for (MGroup& gr : P->groups) {
        if (P->groups.size() > 1) {
            if (cudaStreamCreateWithFlags(&gr.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&gr.join, cudaEventDisableTiming) != cudaSuccess) {
                helios_plan_destroy(P);
                return fail(HELIOS_ECUDA, "stream/event creation failed");
            }
        }
    }
    if (P->groups.size() > 1 && cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming) != cudaSuccess) {
        helios_plan_destroy(P);
        return fail(HELIOS_ECUDA, "event creation failed");
    }
    if ((rc = upload(d_atm, ad)) || (rc = upload(d_tab, td)) || (rc = upload(d_bc, bc)) ||
        (rc = upload(d_items, items)) || (rc = upload(d_order, order)) || (rc = upload(d_gw, gw)) ||
        (rc = upload(d_iP, iP)) || (rc = upload(d_wP, wP)) || (rc = upload(d_dm, dm)) || (rc = upload(d_lnr, lnr)) ||
        (rc = upload(d_lay_atm, lay_atm)) || (rc = upload(d_spec_tab, spec_tab)) || (rc = upload(d_spec_w, spec_w)) ||
        (prm->tabulate && ((rc = upload(d_btab, btab)) || (rc = upload(d_utab, utab))))) {
        helios_plan_destroy(P);
        return rc;
    }
    {
        std::vector<int2> nl(A);
        for (int a = 0; a < A; ++a) nl[a] = make_int2(ad[a].n, ad[a].lay_off);
        if ((rc = upload(P->lay_nl, nl))) {
            helios_plan_destroy(P);
            return rc;
        }
    }
    cudaError_t ce = cudaMemset(dv.warm, 0, std::max<int64_t>(warm, 1) * sizeof(float));
    if (ce == cudaSuccess) ce = cudaMemset(P->counters, 0, sizeof(int) * 2 * kGroups);   // the sweeps keep them at 0
    if (ce != cudaSuccess) { helios_plan_destroy(P); return fail(HELIOS_ECUDA, "cudaMemset: %s", cudaGetErrorString(ce)); }
    dv.atms = d_atm; dv.tabs = d_tab; dv.bins = d_bc; dv.items = d_items; dv.gw = d_gw;
    dv.iP = d_iP; dv.wP = d_wP; dv.dm = d_dm; dv.lnr = d_lnr; dv.lay_atm = d_lay_atm;
    dv.spec_tab = d_spec_tab; dv.spec_w = d_spec_w;
    dv.btab = d_btab; dv.utab = d_utab;
    dv.G = G; dv.TB = TB; dv.A = A; dv.iso_layers = prm->iso_layers;
    dv.dtau_iso = std::max((float)prm->dtau_iso, FLT_MIN);
    dv.D = (float)prm->D; dv.eps = (float)(1.0 / prm->D); dv.w0_pure = (float)prm->w0_pure;
    dv.printed_gradient = prm->printed_gradient;
    P->atms_h = ad;
    P->ws_bytes = (int64_t)tot;
    *out = P;
    return HELIOS_OK;
}

int helios_plan_set_timing(helios_plan* p, int slots)
{
    if (!p) return fail(HELIOS_EINVAL, "helios_plan_set_timing: null plan");
    if (slots < 0 || slots > 65536) return fail(HELIOS_EINVAL, "helios_plan_set_timing: %d slots", slots);
    CUDA_TRY(cudaSetDevice(p->ctx->device));
    CUDA_TRY(cudaDeviceSynchronize());
    for (cudaEvent_t e : p->ev_ring) cudaEventDestroy(e);
    p->ev_ring.clear();
    p->timing = 0;
    p->n_timed = 0;
    for (int i = 0; i < 2 * slots; ++i) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        p->ev_ring.push_back(e);
    }
    p->timing = slots > 0;
    return HELIOS_OK;
}

int helios_plan_sweep_times(helios_plan* p, float* ms, int max_n, int* n_out)
{
    if (!p || !ms || !n_out || max_n < 0) return fail(HELIOS_EINVAL, "helios_plan_sweep_times: bad argument");
    if (!p->timing) return fail(HELIOS_EINVAL, "timing is not enabled on this plan");
    const int64_t slots = (int64_t)p->ev_ring.size() / 2;
    const int64_t avail = std::min<int64_t>(p->n_timed, slots);
    const int64_t n = std::min<int64_t>(avail, max_n);
    for (int64_t k = 0; k < n; ++k) {
        const int64_t idx = (p->n_timed - n + k) % slots;      // oldest of the last n first
        CUDA_TRY(cudaEventSynchronize(p->ev_ring[2 * idx + 1]));
        CUDA_TRY(cudaEventElapsedTime(ms + k, p->ev_ring[2 * idx], p->ev_ring[2 * idx + 1]));
    }
    *n_out = (int)n;
    return HELIOS_OK;
}

int helios_device_recip(const float* x, float* y, int n, cudaStream_t stream)
{
    if (n < 0 || (n > 0 && (!x || !y))) return fail(HELIOS_EINVAL, "helios_device_recip: invalid arguments");
    if (n == 0) return HELIOS_OK;
    recip_kernel<<<(n + 255) / 256, 256, 0, stream>>>(x, y, n);
    CUDA_TRY(cudaGetLastError());
    return HELIOS_OK;
}

int helios_plan_last_sweep_ms(helios_plan* p, float* ms)
{
    int n = 0;
    if (!ms) return fail(HELIOS_EINVAL, "helios_plan_last_sweep_ms: null argument");
    int rc = helios_plan_sweep_times(p, ms, 1, &n);
    if (rc) return rc;
    if (n == 0) return fail(HELIOS_EINVAL, "no timed evaluation yet");
    return HELIOS_OK;
}

// ---- checkpoint of the iteration state a plan keeps between steps: a header (magic, points,
// warm-start floats, layers), the point temperatures of the last evaluation (the old
// temperatures of the next warm-start shift) and the warm-start upward fluxes
constexpr int64_t kStateMagic = 0x4b43534f494c4548LL;     // "HELIOSCK"

static int64_t state_bytes(const helios_plan* p)
{
    return (int64_t)sizeof(p->state_hdr) + (int64_t)sizeof(double) * p->points +
           (int64_t)sizeof(float) * p->warm_floats;
}

int helios_plan_state_bytes(const helios_plan* p, int64_t* bytes)
{
    if (!p || !bytes) return fail(HELIOS_EINVAL, "helios_plan_state_bytes: null argument");
    *bytes = state_bytes(p);
    return HELIOS_OK;
}

int helios_plan_state_export(helios_plan* p, void* buf, cudaStream_t s)
{
    CallRange range_("helios_plan_state_export");
    if (!p || !buf) return fail(HELIOS_EINVAL, "helios_plan_state_export: null argument");
    if (!p->warm_ready) return fail(HELIOS_EINVAL, "helios_plan_state_export: no evaluation has been made yet");
    CUDA_TRY(cudaSetDevice(p->ctx->device));
    p->state_hdr[0] = kStateMagic;
    p->state_hdr[1] = p->points;
    p->state_hdr[2] = p->warm_floats;
    p->state_hdr[3] = p->layers;
    unsigned char* b = static_cast<unsigned char*>(buf);
    CUDA_TRY(cudaMemcpyAsync(b, p->state_hdr, sizeof(p->state_hdr), cudaMemcpyDefault, s));
    b += sizeof(p->state_hdr);
    CUDA_TRY(cudaMemcpyAsync(b, p->dev.Tpt, sizeof(double) * p->points, cudaMemcpyDefault, s));
    b += sizeof(double) * p->points;
    CUDA_TRY(cudaMemcpyAsync(b, p->dev.warm, sizeof(float) * p->warm_floats, cudaMemcpyDefault, s));
    return HELIOS_OK;
}

int helios_plan_state_import(helios_plan* p, const void* buf, cudaStream_t s)
{
    CallRange range_("helios_plan_state_import");
    if (!p || !buf) return fail(HELIOS_EINVAL, "helios_plan_state_import: null argument");
    CUDA_TRY(cudaSetDevice(p->ctx->device));
    CUDA_TRY(cudaStreamSynchronize(s));                  // the checkpoint may still be being written
    int64_t hdr[4];
    CUDA_TRY(cudaMemcpy(hdr, buf, sizeof hdr, cudaMemcpyDefault));
    if (hdr[0] != kStateMagic || hdr[1] != p->points || hdr[2] != p->warm_floats || hdr[3] != p->layers)
        return fail(HELIOS_EINVAL, "helios_plan_state_import: the checkpoint was not made by a plan of this shape");
    const unsigned char* b = static_cast<const unsigned char*>(buf) + sizeof hdr;
    CUDA_TRY(cudaMemcpyAsync(p->dev.Tpt, b, sizeof(double) * p->points, cudaMemcpyDefault, s));
    b += sizeof(double) * p->points;
    CUDA_TRY(cudaMemcpyAsync(p->dev.warm, b, sizeof(float) * p->warm_floats, cudaMemcpyDefault, s));
    p->warm_ready = true;
    return HELIOS_OK;
}

int helios_plan_info(const helios_plan* p, helios_plan_info_t* info)
{
    if (!p || !info) return fail(HELIOS_EINVAL, "helios_plan_info: null argument");
    info->layers = p->layers; info->interfaces = p->interfaces; info->points = p->points;
    info->bins = p->bins; info->cells = p->cells; info->passes = p->passes;
    info->workspace_bytes = p->ws_bytes;
    info->sweep_launches = (int)p->groups.size();
    info->fused_finalize = p->max_items <= kFuseFinalizeItems ? 1 : 0;
    info->warm_floats = p->warm_floats;
    info->spec_floats = p->spec_floats;
    return HELIOS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
namespace {

// the condition of the WHILE node of the radiative-equilibrium graph: loop while any atmosphere is
// active and the chunk budget lasts (the budget bounds the loop whatever the device state)
__global__ void loop_cond_kernel(cudaGraphConditionalHandle h, const int* n_active, int* chunks_left)
{
    const int left = *chunks_left - 1;
    *chunks_left = left;
    cudaGraphSetConditional(h, (*n_active > 0 && left > 0) ? 1u : 0u);
}

// Programmatic dependent launch of the kernels of one evaluation (prep, sweep, finalize, post;
// each waits for its predecessor's completion before touching memory, see pdl_enter): only on
// an ordinary stream -- not while it is being captured into a graph, not between the sweep
// timing events -- and only for plans of a single launch group, whose kernels follow one
// another directly on the caller's stream (with several groups the sweeps run on forked
// streams and rejoin through event waits, so a kernel's predecessor is not always a kernel)
bool use_pdl(const helios_plan* p, cudaStream_t s)
{
    if (p->timing || p->groups.size() != 1) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusNone;
}

template <typename... KArgs, typename... Args>
int launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
    return HELIOS_OK;
}

// optional outputs and buffers of one sweep launch: the emergent spectrum, the per-bin fluxes at
// every point, and a caller-owned warm-start buffer in place of the plan's own
struct SweepIO {
    float* Fup_toa = nullptr;
    float* F_spec = nullptr;
    float* warm = nullptr;
};

template <int M, int MINB, bool DIRECT, int CL = 32>
int launch_sweep_MB(helios_plan* p, const MGroup& gr, const int* status, int n_passes, int warm_valid,
                    const SweepIO& io, cudaStream_t s)
{
    const size_t smem = sweep_smem(M, p->G, CL);
    const int threads = DIRECT ? 32 * p->G : gr.threads;
    static thread_local int configured_dev[kMaxM + 1][4][2][2] = {};      // [M][MINB][DIRECT][16 lanes]
    int& conf = configured_dev[M][MINB][DIRECT][CL == 16];
    if (conf != p->ctx->device + 1) {
        CUDA_TRY(cudaFuncSetAttribute(sweep_kernel<M, MINB, DIRECT, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
        // shared memory for the MINB blocks the registers allow (at G = 20), the rest of the SM's
        // 256 KB stays L1 for the table gathers (batched workload +1%)
        const size_t need = (size_t)MINB * (sweep_smem_bytes(M, 20, CL) + 1024);
        const int pct = (int)std::min<size_t>(100, (100 * need + 228 * 1024 - 1) / (228 * 1024));
        CUDA_TRY(cudaFuncSetAttribute(sweep_kernel<M, MINB, DIRECT, CL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      pct));
        conf = p->ctx->device + 1;
    }
    const bool pdl = use_pdl(p, s);
    PlanDev dv = p->dev;
    if (io.warm) dv.warm = io.warm;
    if (p->prm.persistent)
        return launch_k(pdl, sweep_kernel<M, MINB, DIRECT, CL>, dim3(DIRECT ? gr.grid_direct : gr.grid), dim3(threads),
                        smem, s, dv, (const int*)gr.order, gr.count, gr.counter, status, n_passes, warm_valid,
                        io.Fup_toa, io.F_spec);
    return launch_k(pdl, sweep_kernel<M, MINB, DIRECT, CL>, dim3(gr.count), dim3(threads), smem, s, dv,
                    (const int*)gr.order, gr.count, (int*)nullptr, status, n_passes, warm_valid, io.Fup_toa, io.F_spec);
}

template <int M>
int launch_sweep_M(helios_plan* p, const MGroup& gr, const int* status, int n_passes, int warm_valid,
                   const SweepIO& io, cudaStream_t s)
{
    if constexpr (cl16_chunk(M)) {
        if (gr.cl == 16 && n_passes != HELIOS_DIRECT)
            return launch_sweep_MB<M, minb16<M>(), false, 16>(p, gr, status, n_passes, warm_valid, io, s);
    }
    if (n_passes == HELIOS_DIRECT)
        return launch_sweep_MB<M, sweep_minb<M, true>(), true>(p, gr, status, n_passes, warm_valid, io, s);
    return launch_sweep_MB<M, sweep_minb<M, false>(), false>(p, gr, status, n_passes, warm_valid, io, s);
}

int launch_sweep(helios_plan* p, const int* status, int n_passes, int warm_valid, const SweepIO& io, cudaStream_t s)
{
    if (p->timing) {
        const size_t slot = (size_t)(p->n_timed % (int64_t)(p->ev_ring.size() / 2));
        p->ev_sweep0 = p->ev_ring[2 * slot];
        p->ev_sweep1 = p->ev_ring[2 * slot + 1];
        ++p->n_timed;
        CUDA_TRY(cudaEventRecord(p->ev_sweep0, s));
    }
    const bool fork = p->groups.size() > 1;
    if (fork) CUDA_TRY(cudaEventRecord(p->fork, s));
    for (const MGroup& gr0 : p->groups) {
        int rc = HELIOS_OK;
        const MGroup& gr = gr0;
        cudaStream_t gs = s;
        if (fork) {
            gs = gr.stream;
            CUDA_TRY(cudaStreamWaitEvent(gs, p->fork, 0));
        }
        switch (n_passes == HELIOS_DIRECT ? gr.M_direct : gr.M) {
            case 1: rc = launch_sweep_M<1>(p, gr, status, n_passes, warm_valid, io, gs); break;
            case 3: rc = launch_sweep_M<3>(p, gr, status, n_passes, warm_valid, io, gs); break;
            case 5: rc = launch_sweep_M<5>(p, gr, status, n_passes, warm_valid, io, gs); break;
            case 7: rc = launch_sweep_M<7>(p, gr, status, n_passes, warm_valid, io, gs); break;
            case 9: rc = launch_sweep_M<9>(p, gr, status, n_passes, warm_valid, io, gs); break;
            case 11: rc = launch_sweep_M<11>(p, gr, status, n_passes, warm_valid, io, gs); break;
            case 13: rc = launch_sweep_M<13>(p, gr, status, n_passes, warm_valid, io, gs); break;
            case 15: rc = launch_sweep_M<15>(p, gr, status, n_passes, warm_valid, io, gs); break;
            default: rc = fail(HELIOS_EINVAL, "unsupported lane chunk %d", gr.M);
        }
        if (rc) return rc;
        if (fork) CUDA_TRY(cudaEventRecord(gr.join, gs));
    }
    if (fork)
        for (const MGroup& gr : p->groups) CUDA_TRY(cudaStreamWaitEvent(s, gr.join, 0));
    if (p->timing) CUDA_TRY(cudaEventRecord(p->ev_sweep1, s));
    return HELIOS_OK;
}

int launch_prep(helios_plan* p, const double* T, const int* status, int warm_valid, cudaStream_t s)
{
    return launch_k(use_pdl(p, s), prep_kernel, dim3((2 * p->max_n + 1 + 63) / 64, p->A), dim3(64), 0, s, p->dev, T,
                    status, warm_valid);
}

int launch_eval(helios_plan* p, const double* T, const int* status, int n_passes, int warm_valid, double* Fup,
                double* Fdn, const SweepIO& io, cudaStream_t s)
{
    int rc = launch_prep(p, T, status, warm_valid, s);
    if (rc) return rc;
    rc = launch_sweep(p, status, n_passes, warm_valid, io, s);
    if (rc) return rc;
    return launch_k(use_pdl(p, s), finalize_kernel, dim3(p->max_n + 1, p->A), dim3(32), 0, s, p->dev, status, Fup, Fdn);
}

TempArgs temp_args(const helios_plan* p)
{
    TempArgs t;
    t.sigma = sigmaSB; t.tol = p->prm.tol; t.fpre_num = p->prm.fpre_num; t.fpre_exp = p->prm.fpre_exp;
    t.osc_down = p->prm.osc_down; t.osc_up = p->prm.osc_up; t.mult_max = p->prm.mult_max;
    t.T_floor = p->prm.T_floor; t.max_iter = p->prm.max_iter;
    t.T_tab_max = p->prm.tabulate ? (double)kTabDT * (kTabNT - 1) : 0.0;
    return t;
}

TempArgs temp_args(const helios_plan* p);

// finalize + temperature step (+ the next evaluation's point quantities) of every atmosphere.
// The bolometric sums join the per-atmosphere block when every atmosphere has few work items;
// an atmosphere of many items (a single wide one) keeps them in finalize_kernel: one warp per
// block and interface, so its FP64 sums spread over as many SMs as there are interfaces (the
// FP64 pipe of an SM is narrow)
int launch_post(helios_plan* p, const int* status_gate, double* Fup, double* Fdn, double* T, double* mult,
                uint8_t* hist, uint8_t* nhist, int* status, int* iters, double* metric, int* n_active, int gate,
                int do_prep, cudaStream_t s)
{
    const int fuse = p->max_items <= kFuseFinalizeItems;
    const bool pdl = use_pdl(p, s);
    if (!fuse) {
        const int rc = launch_k(pdl, finalize_kernel, dim3(p->max_n + 1, p->A), dim3(32), 0, s, p->dev, status_gate,
                                Fup, Fdn);
        if (rc) return rc;
    }
    return launch_k(pdl, post_kernel, dim3(p->A), dim3(512), 0, s, p->dev, temp_args(p), Fup, Fdn, T, mult, hist,
                    nhist, status, iters, metric, n_active, gate, fuse, do_prep);
}

int launch_temp(helios_plan* p, const double* Fup, const double* Fdn, double* T, double* mult, uint8_t* hist,
                uint8_t* nhist, int* status, int* iters, double* metric, int* n_active, cudaStream_t s)
{
    const TempArgs ta = temp_args(p);
    const int threads = 32 * ((p->max_n + 31) / 32);          // one block per atmosphere, a thread per layer
    temp_kernel<<<p->A, threads, 0, s>>>(p->dev, ta, Fup, Fdn, T, mult, hist, nhist, status, iters, metric, n_active);
    CUDA_TRY(cudaGetLastError());
    return HELIOS_OK;
}

}  // namespace

extern "C" {

int helios_interp_opacity(helios_plan* p, const double* T_layer, float* kappa_pts, int32_t* idx_pts, double* w_pts,
                          cudaStream_t s)
{
    CallRange range_("helios_interp_opacity");
    if (!p || !T_layer) return fail(HELIOS_EINVAL, "helios_interp_opacity: null argument");
    CUDA_TRY(cudaSetDevice(p->ctx->device));
    long long off = 0;
    for (int a = 0; a < p->A; ++a) {
        const AtmDesc& d = p->atms_h[a];
        const long long total = (long long)(2 * d.n + 1) * d.L * p->G;
        const int blocks = (int)std::min<long long>((total + 255) / 256, 148 * 16);
        interp_kernel<<<blocks, 256, 0, s>>>(p->dev, T_layer, a, kappa_pts, off, idx_pts, w_pts);
        CUDA_TRY(cudaGetLastError());
        off += total;
    }
    return HELIOS_OK;
}

int helios_flux_sweep(helios_plan* p, const double* T_layer, int n_passes, int warm, float* Fup_warm,
                      double* Fup_bol, double* Fdn_bol, float* Fup_toa, float* F_spec, cudaStream_t s)
{
    CallRange range_("helios_flux_sweep");
    if (!p || !T_layer || !Fup_bol || !Fdn_bol) return fail(HELIOS_EINVAL, "helios_flux_sweep: null argument");
    if (Fup_warm && (reinterpret_cast<uintptr_t>(Fup_warm) & 15))
        return fail(HELIOS_EINVAL, "helios_flux_sweep: Fup_warm is not 16-byte aligned");
    if (n_passes < HELIOS_DIRECT) return fail(HELIOS_EINVAL, "helios_flux_sweep: n_passes = %d", n_passes);
    if (n_passes == HELIOS_DIRECT && p->prm.tabulate)
        return fail(HELIOS_EINVAL, "helios_flux_sweep: the exact column solve has no tabulated form");
    if (n_passes == 0) n_passes = p->passes;
    CUDA_TRY(cudaSetDevice(p->ctx->device));
    // a caller-owned warm start is valid when the caller says so; the plan's own once it holds an
    // evaluation.  The shift to the new temperatures uses the point temperatures of this plan's
    // previous evaluation either way
    const int warm_valid = (warm && (Fup_warm || p->warm_ready)) ? 1 : 0;
    SweepIO io;
    io.Fup_toa = Fup_toa;
    io.F_spec = F_spec;
    io.warm = Fup_warm;
    int rc = launch_eval(p, T_layer, nullptr, n_passes, warm_valid, Fup_bol, Fdn_bol, io, s);
    if (rc) return rc;
    if (!Fup_warm) p->warm_ready = true;
    return HELIOS_OK;
}

int helios_temp_update(helios_plan* p, const double* Fup_bol, const double* Fdn_bol, double* T_layer, double* mult,
                       uint8_t* hist, uint8_t* nhist, int32_t* status, int32_t* iters, double* metric, cudaStream_t s)
{
    CallRange range_("helios_temp_update");
    if (!p || !Fup_bol || !Fdn_bol || !T_layer || !mult || !hist || !nhist || !status)
        return fail(HELIOS_EINVAL, "helios_temp_update: null argument");
    CUDA_TRY(cudaSetDevice(p->ctx->device));
    return launch_temp(p, Fup_bol, Fdn_bol, T_layer, mult, hist, nhist, status, iters, metric, nullptr, s);
}

int helios_re_step(helios_plan* p, double* T_layer, int warm, double* mult, uint8_t* hist, uint8_t* nhist,
                   int32_t* status, int32_t* iters, double* metric, double* Fup_bol, double* Fdn_bol, cudaStream_t s)
{
    CallRange range_("helios_re_step");
    if (!p || !T_layer || !mult || !hist || !nhist || !status)
        return fail(HELIOS_EINVAL, "helios_re_step: null argument");
    CUDA_TRY(cudaSetDevice(p->ctx->device));
    const int warm_valid = (warm && p->warm_ready) ? 1 : 0;
    double* Fu = Fup_bol ? Fup_bol : p->Fup;
    double* Fd = Fdn_bol ? Fdn_bol : p->Fdn;
    int rc = launch_prep(p, T_layer, nullptr, warm_valid, s);
    if (!rc) rc = launch_sweep(p, nullptr, p->passes, warm_valid, SweepIO(), s);
    if (!rc) rc = launch_post(p, nullptr, Fu, Fd, T_layer, mult, hist, nhist, status, iters, metric, nullptr, 0, 0, s);
    if (rc) return rc;
    p->warm_ready = true;
    return HELIOS_OK;
}

int helios_re_step_host(helios_plan* p, double* T_host, double* T_dev, int warm, double* mult, uint8_t* hist,
                        uint8_t* nhist, int32_t* status, int32_t* iters, double* metric, int32_t* status_host,
                        cudaStream_t s)
{
    CallRange range_("helios_re_step_host");
    if (!p || !T_host || !T_dev || !status_host) return fail(HELIOS_EINVAL, "helios_re_step_host: null argument");
    CUDA_TRY(cudaSetDevice(p->ctx->device));
    const size_t tb = sizeof(double) * (size_t)p->layers;
    CUDA_TRY(cudaMemcpyAsync(T_dev, T_host, tb, cudaMemcpyHostToDevice, s));
    const int rc = helios_re_step(p, T_dev, warm, mult, hist, nhist, status, iters, metric, nullptr, nullptr, s);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(T_host, T_dev, tb, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(status_host, status, sizeof(int32_t) * (size_t)p->A, cudaMemcpyDeviceToHost, s));
    return HELIOS_OK;
}

int helios_solve_re(helios_plan* p, double* T_layer, int32_t* iters, int32_t* status, cudaStream_t s)
{
    CallRange range_("helios_solve_re");
    if (!p || !T_layer || !iters || !status) return fail(HELIOS_EINVAL, "helios_solve_re: null argument");
    helios_ctx* c = p->ctx;
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t w = c->stream;
    CUDA_TRY(cudaEventRecord(c->ev_in, s));
    CUDA_TRY(cudaStreamWaitEvent(w, c->ev_in, 0));
    // fresh iteration state
    std::vector<double> ones(p->layers, 1.0);
    CUDA_TRY(cudaMemcpyAsync(p->mult, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice, w));
    CUDA_TRY(cudaMemsetAsync(p->hist, 0, p->layers, w));
    CUDA_TRY(cudaMemsetAsync(p->nhist, 0, p->layers, w));
    CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t) * p->A, w));
    CUDA_TRY(cudaMemsetAsync(iters, 0, sizeof(int32_t) * p->A, w));
    const int A = p->A;
    CUDA_TRY(cudaMemcpyAsync(p->n_active, &A, sizeof(int), cudaMemcpyHostToDevice, w));
    const int timing = p->timing;
    p->timing = 0;    // no event records inside the captured graph
    struct Restore { helios_plan* p; int t; ~Restore() { p->timing = t; } } restore{p, timing};
    // first temperature step: the coupled stream starts from zero.  Every step ends with
    // post_kernel, which also prepares the next evaluation at the new temperatures
    int rc = launch_prep(p, T_layer, status, 0, w);
    if (!rc) rc = launch_sweep(p, status, p->passes, 0, SweepIO(), w);
    if (!rc) rc = launch_post(p, status, p->Fup, p->Fdn, T_layer, p->mult, p->hist, p->nhist, status, iters, nullptr,
                              p->n_active, 1, 1, w);
    if (rc) return rc;
    // later steps start from the previous step's fluxes; captured as a graph of `chunk` steps,
    // either inside a conditional WHILE node that the device keeps looping (device_loop) or
    // relaunched by the host between reads of the active count
    const int chunk = p->prm.check_every > 0 ? p->prm.check_every : 16;
    const int dloop = p->prm.device_loop;
    const void* key[3] = {T_layer, iters, status};
    if (!p->graph || p->graph_chunk != chunk || p->graph_device_loop != dloop ||
        std::memcmp(key, p->graph_key, sizeof key) != 0) {
        if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
        cudaGraph_t g = nullptr;
        cudaGraphConditionalHandle h = 0;
        if (dloop) {
            CUDA_TRY(cudaGraphCreate(&g, 0));
            // zero-filled storage: the parameter union has no default constructor
            alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)] = {};
            cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_raw);
            cudaGraphNode_t node;
            cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
            if (e == cudaSuccess) {
                np.type = cudaGraphNodeTypeConditional;
                np.conditional.handle = h;
                np.conditional.type = cudaGraphCondTypeWhile;
                np.conditional.size = 1;
                e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
            }
            if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(w, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                                   cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                cudaGraphDestroy(g);
                return fail(HELIOS_ECUDA, "conditional graph: %s", cudaGetErrorString(e));
            }
        } else {
            CUDA_TRY(cudaStreamBeginCapture(w, cudaStreamCaptureModeThreadLocal));
        }
        for (int i = 0; i < chunk && rc == HELIOS_OK; ++i) {
            rc = launch_sweep(p, status, p->passes, 1, SweepIO(), w);
            if (rc == HELIOS_OK)
                rc = launch_post(p, status, p->Fup, p->Fdn, T_layer, p->mult, p->hist, p->nhist, status, iters,
                                 nullptr, p->n_active, 1, 1, w);
        }
        if (rc == HELIOS_OK && dloop) {
            loop_cond_kernel<<<1, 1, 0, w>>>(h, p->n_active, p->chunks_left);
            if (cudaGetLastError() != cudaSuccess) rc = fail(HELIOS_ECUDA, "loop condition launch failed");
        }
        cudaGraph_t captured = nullptr;
        cudaError_t ec = cudaStreamEndCapture(w, &captured);
        if (!dloop) g = captured;
        if (rc || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc ? rc : fail(HELIOS_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
        }
        cudaError_t ei = cudaGraphInstantiate(&p->graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) { p->graph = nullptr; return fail(HELIOS_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei)); }
        std::memcpy(p->graph_key, key, sizeof key);
        p->graph_chunk = chunk;
        p->graph_device_loop = dloop;
    }
    // the kernel itself retires atmospheres at max_iter; the chunk budget is only a backstop
    const int budget = (p->prm.max_iter + chunk - 1) / chunk + 1;
    if (dloop) {
        CUDA_TRY(cudaMemcpyAsync(p->chunks_left, &budget, sizeof(int), cudaMemcpyHostToDevice, w));
        CUDA_TRY(cudaGraphLaunch(p->graph, w));
    } else {
        for (int k = 0; k < budget; ++k) {
            CUDA_TRY(cudaGraphLaunch(p->graph, w));
            CUDA_TRY(cudaMemcpyAsync(c->h_active, p->n_active, sizeof(int), cudaMemcpyDeviceToHost, w));
            CUDA_TRY(cudaStreamSynchronize(w));
            if (*c->h_active <= 0) break;
        }
    }
    p->warm_ready = true;
    CUDA_TRY(cudaEventRecord(c->ev_out, w));
    CUDA_TRY(cudaStreamWaitEvent(s, c->ev_out, 0));
    std::vector<int32_t> st(A);
    CUDA_TRY(cudaMemcpyAsync(st.data(), status, sizeof(int32_t) * A, cudaMemcpyDeviceToHost, w));
    CUDA_TRY(cudaStreamSynchronize(w));
    for (int a = 0; a < A; ++a)
        if (st[a] != HELIOS_ATM_CONVERGED)
            return fail(HELIOS_ENOCONV, "atmosphere %d ended with status %d", a, st[a]);
    return HELIOS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: times one flux evaluation of a calibration subset of the batch for each
// candidate work-item size and launch mode; caches the winner per (device, shape bucket).
namespace {

std::string shape_key(const helios_batch_t* b, int G, const char* dev_name)
{
    double mn = 0.0, mL = 0.0;
    bool scat = false;
    int64_t off = 0;
    for (int a = 0; a < b->A; ++a) {
        mn += b->n_layers[a];
        mL += b->n_bins[a];
        for (int l = 0; l < b->n_bins[a]; ++l) scat |= b->omega0[off + l] != 0.0f;
        off += b->n_bins[a];
    }
    mn /= b->A;
    mL /= b->A;
    int lgA = 0;
    while ((1 << (lgA + 1)) <= b->A) ++lgA;
    char buf[384];
    snprintf(buf, sizeof buf, "%s|A2^%d|n%d|L%d|G%d|%s", dev_name, lgA, (int)(mn / 25.0 + 0.5) * 25,
             (int)(mL / 250.0 + 0.5) * 250, G, scat ? "scat" : "abs");
    return buf;
}

bool cache_lookup(const char* path, const std::string& key, int& tb, int& pers)
{
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    std::string txt;
    char buf[4096];
    size_t r;
    while ((r = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, r);
    fclose(f);
    const std::string pat = "\"" + key + "\": {";
    const size_t at = txt.find(pat);
    if (at == std::string::npos) return false;
    return sscanf(txt.c_str() + at + pat.size(), " \"bins_per_item\": %d, \"persistent\": %d", &tb, &pers) == 2;
}

void cache_store(const char* path, const std::string& key, int tb, int pers, double ms)
{
    if (!path) return;
    std::string txt;
    if (FILE* f = fopen(path, "r")) {
        char buf[4096];
        size_t r;
        while ((r = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, r);
        fclose(f);
    }
    const size_t close = txt.rfind('}');
    char entry[640];
    snprintf(entry, sizeof entry, "\"%s\": {\"bins_per_item\": %d, \"persistent\": %d, \"ms\": %.6f}", key.c_str(), tb,
             pers, ms);
    std::string out;
    if (close == std::string::npos || txt.find('{') == std::string::npos) out = std::string("{\n  ") + entry + "\n}\n";
    else out = txt.substr(0, close) + (txt.find('"') != std::string::npos ? ",\n  " : "  ") + entry + "\n}\n";
    const std::string tmp = std::string(path) + ".tmp";
    if (FILE* f = fopen(tmp.c_str(), "w")) {
        fwrite(out.data(), 1, out.size(), f);
        fclose(f);
        rename(tmp.c_str(), path);
    }
}

}  // namespace

extern "C" int helios_autotune(helios_ctx* ctx, const helios_batch_t* b, const helios_ktable_t* tabs, int ntab,
                               const helios_params_t* base, const char* cache_path, helios_params_t* tuned)
{
    CallRange range_("helios_autotune");
    if (!ctx || !b || !tabs || !base || !tuned || b->A < 1 || ntab < 1)
        return fail(HELIOS_EINVAL, "helios_autotune: bad argument");
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, ctx->device));
    const std::string key = shape_key(b, tabs[0].G, prop.name);
    *tuned = *base;
    int tb = 0, pers = 0;
    if (cache_lookup(cache_path, key, tb, pers)) {
        tuned->bins_per_item = tb;
        tuned->persistent = pers;
        return HELIOS_OK;
    }
    // calibration subset: up to 128 atmospheres spread over the batch
    const int stride = std::max(1, b->A / 128);
    std::vector<int32_t> n, L, tid;
    std::vector<double> Pt, Pb, gr, Ti, Tn, Ts, nu;
    std::vector<float> w0, g0;
    std::vector<int64_t> nu_off(b->A + 1, 0), bin_off(b->A + 1, 0);
    for (int a = 0; a < b->A; ++a) {
        nu_off[a + 1] = nu_off[a] + b->n_bins[a] + 1;
        bin_off[a + 1] = bin_off[a] + b->n_bins[a];
    }
    int64_t layers = 0;
    for (int a = 0; a < b->A; a += stride) {
        n.push_back(b->n_layers[a]); L.push_back(b->n_bins[a]); tid.push_back(b->table_id[a]);
        Pt.push_back(b->P_top_bar[a]); Pb.push_back(b->P_bot_bar[a]); gr.push_back(b->grav[a]);
        Ti.push_back(b->T_irr[a]); Tn.push_back(b->T_int[a]); Ts.push_back(b->T_star[a]);
        nu.insert(nu.end(), b->nu_edges + nu_off[a], b->nu_edges + nu_off[a + 1]);
        w0.insert(w0.end(), b->omega0 + bin_off[a], b->omega0 + bin_off[a + 1]);
        g0.insert(g0.end(), b->g0 + bin_off[a], b->g0 + bin_off[a + 1]);
        layers += b->n_layers[a];
    }
    helios_batch_t sub;
    sub.A = (int)n.size(); sub.n_layers = n.data(); sub.n_bins = L.data(); sub.table_id = tid.data();
    sub.P_top_bar = Pt.data(); sub.P_bot_bar = Pb.data(); sub.grav = gr.data(); sub.T_irr = Ti.data();
    sub.T_int = Tn.data(); sub.T_star = Ts.data(); sub.nu_edges = nu.data(); sub.omega0 = w0.data(); sub.g0 = g0.data();
    sub.species_off = nullptr; sub.species_table = nullptr; sub.species_weight = nullptr;   // timing only
    double *dT = nullptr, *dFu = nullptr, *dFd = nullptr;
    int64_t ifc = layers + sub.A;
    if (cudaMalloc((void**)&dT, sizeof(double) * layers) != cudaSuccess ||
        cudaMalloc((void**)&dFu, sizeof(double) * ifc) != cudaSuccess ||
        cudaMalloc((void**)&dFd, sizeof(double) * ifc) != cudaSuccess) {
        cudaFree(dT); cudaFree(dFu); cudaFree(dFd);
        return fail(HELIOS_ENOMEM, "helios_autotune: scratch allocation failed");
    }
    std::vector<double> T0(layers, 1000.0);
    cudaMemcpy(dT, T0.data(), sizeof(double) * layers, cudaMemcpyHostToDevice);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    int best_tb = 1, best_p = 1, rc = HELIOS_OK;
    const int cands[] = {1, 2, 4, 8, 16, 32};
    for (int pm = 0; pm <= 1 && rc == HELIOS_OK; ++pm)
        for (int c : cands) {
            helios_params_t p = *base;
            p.bins_per_item = c;
            p.persistent = pm;
            helios_plan* plan = nullptr;
            rc = helios_plan_create(ctx, &sub, tabs, ntab, &p, &plan);
            if (rc) break;
            float ms[3];
            rc = helios_flux_sweep(plan, dT, 0, 0, nullptr, dFu, dFd, nullptr, nullptr, ctx->stream);
            for (int r = 0; r < 3 && rc == HELIOS_OK; ++r) {
                cudaEventRecord(e0, ctx->stream);
                rc = helios_flux_sweep(plan, dT, 0, 1, nullptr, dFu, dFd, nullptr, nullptr, ctx->stream);
                cudaEventRecord(e1, ctx->stream);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms[r], e0, e1);
            }
            helios_plan_destroy(plan);
            if (rc) break;
            std::sort(ms, ms + 3);
            if (ms[1] < best) { best = ms[1]; best_tb = c; best_p = pm; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dT); cudaFree(dFu); cudaFree(dFd);
    if (rc) return rc;
    tuned->bins_per_item = best_tb;
    tuned->persistent = best_p;
    cache_store(cache_path, key, best_tb, best_p, best);
    return HELIOS_OK;
}
