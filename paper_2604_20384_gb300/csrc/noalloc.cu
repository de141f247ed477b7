// hvp_hvp_noalloc: loss, gradient and HVP for callers that must not allocate
// device memory (a framework whose allocator owns the device pool, a process
// under a hard device-memory budget). The call is synchronous: it uploads its
// tables from host memory and waits for its stream before returning.
//
// It runs the existing single-window schedule (one tile of 2^n amplitudes per
// sample, n <= 12): FP64 gate preparation, one window pass that goes forward
// through every gate and back again, and the FP64 post-processing. Everything
// those kernels need beyond the caller's inputs and outputs (gate tables,
// FP32 copies of the inputs, per-sample environment records, status word)
// lives in one static device array, so the call allocates nothing.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/hvp.h"
#include "internal.h"
#include "nvtx.h"

namespace hvp {
namespace {

// The work space. Every GPU that loads the library holds it until exit.
__device__ __align__(256) unsigned char g_noalloc_scratch[HVP_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (the symbol name is only a host-side stand-in).
std::mutex g_mu;
void* g_addr[128] = {};
bool g_limits_set[128] = {};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t pass, gates, mats, psi1q, phi, pos, partial, env, T, Om, gr, hr, ge_sink, he_sink, loss_sink, status, total;
};

Layout layout_for(int n, int K, int ns) {
    Layout l{};
    size_t o = 0;
    l.pass = o;    o = align256(o + sizeof(DevPass));
    l.gates = o;   o = align256(o + sizeof(DevGate) * (size_t)K);
    l.mats = o;    o = align256(o + sizeof(Mats32) * (size_t)K);
    l.psi1q = o;   o = align256(o + sizeof(float2) * 2 * (size_t)n * ns);
    l.phi = o;     o = align256(o + sizeof(float2) * ((size_t)1 << n) * ns);
    l.pos = o;     o = align256(o + sizeof(int) * (size_t)n);
    l.partial = o; o = align256(o + 64 * sizeof(double) * (size_t)K * ns);
    l.env = o;     o = align256(o + 64 * sizeof(double) * (size_t)K * ns);
    l.T = o;       o = align256(o + sizeof(double2) * (size_t)ns);
    l.Om = o;      o = align256(o + sizeof(double2) * (size_t)ns);
    l.gr = o;      o = align256(o + sizeof(double2) * 16 * (size_t)K);
    l.hr = o;      o = align256(o + sizeof(double2) * 16 * (size_t)K);
    l.ge_sink = o; o = align256(o + sizeof(double2) * 16 * (size_t)K);   // outputs the caller did not ask for
    l.he_sink = o; o = align256(o + sizeof(double2) * 16 * (size_t)K);
    l.loss_sink = o; o = align256(o + sizeof(double));
    l.status = o;  o = align256(o + sizeof(int));
    l.total = o;
    return l;
}

int err(int code, const char* msg) {
    set_thread_error(msg);
    return code;
}

#define NA_TRY(call)                                                                             \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            char b_[256];                                                                        \
            snprintf(b_, sizeof b_, "hvp_hvp_noalloc: %s: %s", #call, cudaGetErrorString(e_));   \
            return err(HVP_ECUDA, b_);                                                           \
        }                                                                                        \
    } while (0)

}  // namespace
}  // namespace hvp

using namespace hvp;

extern "C" int hvp_hvp_noalloc(int n, int n_layers, int n_samples, const double* psi_1q_dev,
                               const double* phi_dev, const double* G_dev, const double* V_dev,
                               double* loss_dev, double* grad_dev, double* hvp_dev, void* stream) {
    NvtxRange range("hvp_hvp_noalloc");
    if (!psi_1q_dev || !phi_dev || !G_dev) return err(HVP_EINVAL, "hvp_hvp_noalloc: NULL input pointer");
    if (n < 2 || n > 12) return err(HVP_EINVAL, "hvp_hvp_noalloc: n must be in [2, 12]");
    if (n_layers < 1 || n_samples < 1) return err(HVP_EINVAL, "hvp_hvp_noalloc: n_layers and n_samples must be >= 1");
    const int K = num_gates(n, n_layers);
    if (K > kMaxGatesPerPass) return err(HVP_EINVAL, "hvp_hvp_noalloc: more than 64 gates");
    const Layout lay = layout_for(n, K, n_samples);
    if (lay.total > (size_t)HVP_NOALLOC_SCRATCH_BYTES) {
        char b[200];
        snprintf(b, sizeof b, "hvp_hvp_noalloc: needs %zu bytes of work space, the static array holds %u",
                 lay.total, (unsigned)HVP_NOALLOC_SCRATCH_BYTES);
        return err(HVP_EINVAL, b);
    }
    const bool tan = V_dev != nullptr;
    cudaStream_t st = (cudaStream_t)stream;

    // One-time set-up per device: the array's device address.
    int dev = 0;
    NA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return err(HVP_EINVAL, "hvp_hvp_noalloc: device ordinal out of range");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            NA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            g_addr[dev] = p;
        }
        if (!g_limits_set[dev]) {
            NA_TRY(tiled_set_smem_limits());
            g_limits_set[dev] = true;
        }
        base = static_cast<unsigned char*>(g_addr[dev]);
    }

    // Plan: one window over all n qubits (standard layout), every gate in it.
    Plan plan;
    if (make_plan(n, n_layers, n, std::min(kLowBits, n - 1), plan) != HVP_OK || plan.passes.size() != 1)
        return err(HVP_EINVAL, "hvp_hvp_noalloc: the circuit does not fit one window pass");
    std::vector<DevPass> dp;
    std::vector<DevGate> dg;
    build_dev_passes(plan, dp, dg);
    // phi (given in the standard layout) goes into the layout in which the
    // single pass reads its co-states
    int pos[32];
    for (int q = 0; q < n; ++q) pos[q] = plan.passes[0].pos_in[q];

    DevPass* d_pass = reinterpret_cast<DevPass*>(base + lay.pass);
    DevGate* d_gates = reinterpret_cast<DevGate*>(base + lay.gates);
    Mats32* d_mats = reinterpret_cast<Mats32*>(base + lay.mats);
    float2* d_psi = reinterpret_cast<float2*>(base + lay.psi1q);
    float2* d_phi = reinterpret_cast<float2*>(base + lay.phi);
    int* d_pos = reinterpret_cast<int*>(base + lay.pos);
    double* d_partial = reinterpret_cast<double*>(base + lay.partial);
    double* d_env = reinterpret_cast<double*>(base + lay.env);
    int* d_status = reinterpret_cast<int*>(base + lay.status);

    // The array keeps the previous call's contents: the status word must start
    // at zero; every other region is fully rewritten below before it is read.
    NA_TRY(cudaMemcpyAsync(d_pass, dp.data(), sizeof(DevPass), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_gates, dg.data(), sizeof(DevGate) * dg.size(), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(d_pos, pos, sizeof(int) * n, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), st));
    NA_TRY(launch_psi1q_convert(psi_1q_dev, d_psi, (size_t)n_samples * n * 2, st));
    NA_TRY(launch_phi_permute(reinterpret_cast<const double2*>(phi_dev), d_phi, false, n, n_samples, d_pos, st));
    NA_TRY(launch_prep(reinterpret_cast<const double2*>(G_dev), reinterpret_cast<const double2*>(V_dev), d_mats,
                       false, K, d_status, st));

    TiledArgs a{};
    a.pass = d_pass;
    a.gates = d_gates;
    a.mats = d_mats;
    a.psi1q = d_psi;
    a.phi = d_phi;
    a.partial = d_partial;
    a.n = n;
    a.n_samples = n_samples;
    a.mode = M_GEN | M_FWD | M_BWD | M_LOAD_PHI;
    a.tiles_per_cta = 1;
    a.cx_count = 1;
    NA_TRY(launch_tiled(a, tan, n, 256, std::max(K, 1), st));

    PostArgs p{};
    p.partial = d_partial;
    p.env = d_env;
    p.G = reinterpret_cast<const double2*>(G_dev);
    p.V = reinterpret_cast<const double2*>(V_dev);
    p.T = reinterpret_cast<double2*>(base + lay.T);
    p.Omega = reinterpret_cast<double2*>(base + lay.Om);
    p.loss = loss_dev ? loss_dev : reinterpret_cast<double*>(base + lay.loss_sink);
    p.grad_e = grad_dev ? reinterpret_cast<double2*>(grad_dev) : reinterpret_cast<double2*>(base + lay.ge_sink);
    p.hvp_e = hvp_dev ? reinterpret_cast<double2*>(hvp_dev) : reinterpret_cast<double2*>(base + lay.he_sink);
    p.grad_r = reinterpret_cast<double2*>(base + lay.gr);
    p.hvp_r = reinterpret_cast<double2*>(base + lay.hr);
    p.K = K;
    p.n_samples = n_samples;
    p.cx_count = 1;
    p.tangent = tan ? 1 : 0;
    NA_TRY(launch_post(p, st));

    int status = 0;
    NA_TRY(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    if (status) return err(HVP_ENONFINITE, "hvp_hvp_noalloc: a gate is singular or not finite");
    return HVP_OK;
}
