// Allocation-free single-atmosphere flux evaluation: helios_flux_sweep_noalloc.
//
// Who needs this: callers that must not allocate device memory themselves or through
// a library -- code running under a framework that owns the whole device pool, code
// inside a region where allocation is forbidden, or tools that bound their footprint
// up front.  helios_plan_create allocates its workspace with cudaMalloc; this entry
// point instead works out of one fixed scratch array that lives in this file as a
// static __device__ object, so the call itself allocates nothing, on the device or on
// the host.
//
// Cost of that choice: every GPU on which the library's code runs holds the
// kScratchBytes array until the process exits, the array is shared by every call (so
// calls whose GPU work overlaps race on it), and sizes beyond what fits are rejected.
// The host-side staging arrays are static too and are guarded by a mutex.  The host set-up
// (grid, Gauss weights, per-bin constants) is the plan's own (helios_setup.h).
#include "helios.h"

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

// this file's own copy of the device kernels (a separate module, so its static scratch
// array is only loaded on devices that use this entry point)
namespace noalloc_copy {
#include "helios_kernels.cuh"
#include "helios_setup.h"
}
using namespace noalloc_copy::helios_dev;
using namespace noalloc_copy::helios_setup;

// defined with the rest of the error handling in helios_api.cu (not exported)
__attribute__((visibility("hidden"))) void helios_set_error_text(const char* msg);

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;    // 64 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kMaxN = 239;                            // lane chunk M <= 15
constexpr int kMaxNP = 2 * kMaxN + 1;
constexpr int kMaxL = 8192;
constexpr int kMaxG = 20;

// the scratch: file-scope, device-resident; host code only ever sees its symbol
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};                // device address of g_scratch, per device
bool g_smem_set[kMaxDevices][kMaxDevices] = {};       // [device][M] dynamic-smem attribute set

// static host staging (no heap)
AtmDesc h_atm;
TabDesc h_tab;
BinConst h_bins[kMaxL];
int2 h_items[kMaxL];
int h_order[kMaxL];
float h_gw[kMaxG];
int h_iP[kMaxNP];
double h_wP[kMaxNP];
float h_dm[2 * kMaxN];
double h_lnr[kMaxN];
int h_lay_atm[kMaxN];
double h_P[kMaxNP];

int err(int code, const char* fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    helios_set_error_text(msg);            // reported by helios_last_error()
    return code;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Carve {
    char* base;
    size_t off;
    template <typename T>
    T* take(size_t count)
    {
        T* p = reinterpret_cast<T*>(base + off);
        off = align256(off + std::max<size_t>(count, 1) * sizeof(T));
        return p;
    }
};

#define NA_CUDA(call)                                                                                 \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return err(HELIOS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

template <int M>
int launch_sweep(const PlanDev& P, int dev, int count, const int* order, int n_passes, float* toa, cudaStream_t s)
{
    constexpr int MINB = sweep_minb<M, false>();
    const size_t smem = sweep_smem_bytes(M, P.G);
    if (!g_smem_set[dev][M]) {
        NA_CUDA(cudaFuncSetAttribute(sweep_kernel<M, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        g_smem_set[dev][M] = true;
    }
    sweep_kernel<M, MINB><<<count, sweep_block_threads(P.G, false), smem, s>>>(P, order, count, nullptr, nullptr,
                                                                              n_passes, 0, toa, nullptr);
    NA_CUDA(cudaGetLastError());
    return HELIOS_OK;
}

}  // namespace

extern "C" int helios_flux_sweep_noalloc(const helios_batch_t* b, const helios_ktable_t* tab,
                                         const helios_params_t* prm, const double* T_layer, int n_passes,
                                         double* Fup_bol, double* Fdn_bol, float* Fup_toa, cudaStream_t s)
{
    if (!b || !tab || !prm || !T_layer || !Fup_bol || !Fdn_bol)
        return err(HELIOS_EINVAL, "helios_flux_sweep_noalloc: null argument");
    if (b->A != 1) return err(HELIOS_EINVAL, "helios_flux_sweep_noalloc: one atmosphere per call (got %d)", b->A);
    {
        // the call stages its inputs from static host arrays with pageable copies, which a graph
        // cannot capture (and a replay would read whatever a later call left there)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        NA_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return err(HELIOS_EINVAL, "helios_flux_sweep_noalloc: the stream is capturing a graph");
    }
    const int n = b->n_layers[0], L = b->n_bins[0], G = tab->G;
    if (n < 2 || n > kMaxN) return err(HELIOS_EINVAL, "n_layers %d outside [2, %d]", n, kMaxN);
    if (L < 1 || L > kMaxL || L > tab->L) return err(HELIOS_EINVAL, "n_bins %d outside [1, min(%d, table)]", L, kMaxL);
    if (G < 1 || G > kMaxG) return err(HELIOS_EINVAL, "G %d outside [1, %d]", G, kMaxG);
    if (!tab->kappa || ((uintptr_t)tab->kappa & 15) || tab->nP < 1 || tab->nT < 1)
        return err(HELIOS_EINVAL, "invalid k-table");
    if ((int64_t)tab->nP * tab->nT * tab->L * G >= ((int64_t)1 << 31)) return err(HELIOS_EINVAL, "k-table too large");
    if (!(b->P_top_bar[0] > 0.0) || !(b->P_bot_bar[0] > b->P_top_bar[0]) || !(b->grav[0] > 0.0) ||
        !(b->T_irr[0] >= 0.0) || !(b->T_int[0] >= 0.0) || !(b->T_star[0] > 0.0))
        return err(HELIOS_EINVAL, "invalid pressure range, gravity or temperatures");
    if (prm->grey_mode && L != 2) return err(HELIOS_EINVAL, "grey mode needs 2 bins");
    if (prm->iso_layers) return err(HELIOS_EINVAL, "isothermal layers are not supported without a plan");
    for (int l = 0; l <= L; ++l)
        if (!(b->nu_edges[l] > 0.0) || (l > 0 && !(b->nu_edges[l] > b->nu_edges[l - 1])))
            return err(HELIOS_EINVAL, "bin edges must be positive and increasing");
    for (int l = 0; l < L; ++l) {
        const float w0 = b->omega0[l], g0 = b->g0[l];
        if (!(w0 >= 0.0f && w0 <= 1.0f) || !(g0 >= -1.0f && g0 <= 1.0f) ||
            (!(1.0 - (double)w0 < prm->w0_pure) && !(w0 < 1.0f)))
            return err(HELIOS_EINVAL, "bin %d: omega0 %g / g0 %g invalid", l, w0, g0);
    }
    int M = (2 * n + 1 + 31) / 32;
    if (!(M & 1)) ++M;
    int dev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return err(HELIOS_EINVAL, "device %d beyond %d", dev, kMaxDevices);

    std::lock_guard<std::mutex> lock(g_mu);
    // once per device, with that device current: the device address of the scratch array
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        NA_CUDA(cudaGetSymbolAddress(&ptr, g_scratch));
        g_scratch_ptr[dev] = ptr;
    }
    int nsm = 148;
    NA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int per_sm = M <= 7 ? 2 : 1;
    const int TB = prm->bins_per_item > 0 ? prm->bins_per_item
                                          : std::max(1, std::min(32, (L + nsm * per_sm - 1) / (nsm * per_sm)));
    const int items = (L + TB - 1) / TB;
    const int NP = 2 * n + 1, NS = 2 * n;

    // carve the scratch; reject what does not fit before touching the GPU
    Carve c{static_cast<char*>(g_scratch_ptr[dev]), 0};
    PlanDev P;
    std::memset(&P, 0, sizeof P);
    AtmDesc* d_atm = c.take<AtmDesc>(1);
    TabDesc* d_tab = c.take<TabDesc>(1);
    BinConst* d_bins = c.take<BinConst>(L);
    int2* d_items = c.take<int2>(items);
    int* d_order = c.take<int>(items);
    float* d_gw = c.take<float>(G);
    int* d_iP = c.take<int>(NP);
    double* d_wP = c.take<double>(NP);
    float* d_dm = c.take<float>(NS);
    double* d_lnr = c.take<double>(n);
    int* d_lay = c.take<int>(n);
    P.Tpt = c.take<double>(NP); P.iT = c.take<int>(NP); P.wT = c.take<double>(NP); P.row = c.take<int>(NP);
    P.wq = c.take<float4>(NP); P.invT = c.take<float2>(NP); P.Tf = c.take<float>(NP);
    P.invT_old = c.take<float2>(NP); P.dinv_step = c.take<float>(NP); P.dT_step = c.take<float>(NP);
    P.dinv_sub = c.take<float>(NS); P.dT_sub = c.take<float>(NS);
    P.part = c.take<double>((size_t)items * 3 * (n + 1));
    P.warm = nullptr;                      // a cold start stores no warm start
    if (c.off > kScratchBytes)
        return err(HELIOS_EINVAL, "atmosphere needs %zu bytes of scratch, more than the %zu available", c.off,
                   kScratchBytes);

    // ---- host set-up into the static staging arrays (double precision), as helios_plan_create
    layer_geometry(n, b->P_bot_bar[0], b->P_top_bar[0], b->grav[0], 0, *tab, h_P, h_iP, h_wP, h_dm, h_lnr);
    for (int i = 0; i < n; ++i) h_lay_atm[i] = 0;
    const bool any_scat = bin_constants(b->nu_edges, b->omega0, b->g0, L, b->T_irr[0], b->T_int[0], b->T_star[0],
                                        *prm, h_bins);
    if (n_passes < 0) return err(HELIOS_EINVAL, "n_passes = %d (the direct column solve needs a plan)", n_passes);
    if (prm->direct) return err(HELIOS_EINVAL, "the direct column solve needs a plan");
    if (prm->rayleigh) return err(HELIOS_EINVAL, "Rayleigh scattering needs a plan");
    if (prm->tabulate) return err(HELIOS_EINVAL, "tabulated functions need a plan");
    if (n_passes == 0) n_passes = any_scat ? 1 + prm->n_scat : 1;
    for (int t = 0; t < items; ++t) { h_items[t] = make_int2(0, t); h_order[t] = t; }
    gauss_weights01(G, h_gw);
    std::memset(&h_atm, 0, sizeof h_atm);
    h_atm.n = n; h_atm.L = L; h_atm.M = M; h_atm.cl = 32; h_atm.tab = 0; h_atm.n_items = items;
    std::memset(&h_tab, 0, sizeof h_tab);
    h_tab.kappa = tab->kappa; h_tab.nP = tab->nP; h_tab.nT = tab->nT; h_tab.L = tab->L; h_tab.G = G;
    h_tab.log10P0 = tab->log10P0; h_tab.dlog10P = tab->dlog10P; h_tab.T0 = tab->T0; h_tab.dT = tab->dT;
    h_tab.rowL = tab->L * G;
    h_tab.offP = tab->nP > 1 ? tab->nT * h_tab.rowL : 0;
    h_tab.offT = tab->nT > 1 ? h_tab.rowL : 0;

    // ---- stage into the scratch (pageable copies: each returns once the source is consumed)
    NA_CUDA(cudaMemcpyAsync(d_atm, &h_atm, sizeof h_atm, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_tab, &h_tab, sizeof h_tab, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_bins, h_bins, sizeof(BinConst) * L, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_items, h_items, sizeof(int2) * items, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_order, h_order, sizeof(int) * items, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_gw, h_gw, sizeof(float) * G, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_iP, h_iP, sizeof(int) * NP, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_wP, h_wP, sizeof(double) * NP, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_dm, h_dm, sizeof(float) * NS, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_lnr, h_lnr, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    NA_CUDA(cudaMemcpyAsync(d_lay, h_lay_atm, sizeof(int) * n, cudaMemcpyHostToDevice, s));
    P.atms = d_atm; P.tabs = d_tab; P.bins = d_bins; P.items = d_items; P.gw = d_gw; P.iP = d_iP; P.wP = d_wP;
    P.dm = d_dm; P.lnr = d_lnr; P.lay_atm = d_lay;
    P.G = G; P.TB = TB; P.A = 1; P.dtau_iso = std::max((float)prm->dtau_iso, FLT_MIN);

    // ---- one cold-start evaluation: nothing in the scratch is read before this call writes it
    prep_kernel<<<dim3((NP + 63) / 64, 1), 64, 0, s>>>(P, T_layer, nullptr, 0);
    NA_CUDA(cudaGetLastError());
    int rc = HELIOS_OK;
    switch (M) {
        case 1: rc = launch_sweep<1>(P, dev, items, d_order, n_passes, Fup_toa, s); break;
        case 3: rc = launch_sweep<3>(P, dev, items, d_order, n_passes, Fup_toa, s); break;
        case 5: rc = launch_sweep<5>(P, dev, items, d_order, n_passes, Fup_toa, s); break;
        case 7: rc = launch_sweep<7>(P, dev, items, d_order, n_passes, Fup_toa, s); break;
        case 9: rc = launch_sweep<9>(P, dev, items, d_order, n_passes, Fup_toa, s); break;
        case 11: rc = launch_sweep<11>(P, dev, items, d_order, n_passes, Fup_toa, s); break;
        case 13: rc = launch_sweep<13>(P, dev, items, d_order, n_passes, Fup_toa, s); break;
        case 15: rc = launch_sweep<15>(P, dev, items, d_order, n_passes, Fup_toa, s); break;
        default: rc = err(HELIOS_EINVAL, "unsupported lane chunk %d", M);
    }
    if (rc) return rc;
    finalize_kernel<<<dim3((n + 1 + 7) / 8, 1), 256, 0, s>>>(P, nullptr, Fup_bol, Fdn_bol);
    NA_CUDA(cudaGetLastError());
    return HELIOS_OK;
}
