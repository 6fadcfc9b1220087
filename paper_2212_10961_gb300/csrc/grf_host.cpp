// Host side of the C ABI (include/grf.h): argument checking, error reporting,
// the counter-based generator and mode drawing (S1), packing of the device
// mode table, the plan registry, and dispatch to the CUDA launchers.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "grf_internal.h"

namespace grf {

// ---------------------------------------------------------------------------
// Errors and counters
// ---------------------------------------------------------------------------
namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(int err, const char* what) {
    return fail(GRF_ECUDA, "%s: %s", what, cudaGetErrorString(static_cast<cudaError_t>(err)));
}

bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

std::atomic<int32_t> g_inject_alloc{0};  // host allocation failures still to inject

// Maps an exception thrown below an ABI entry point to a status code: no
// exception crosses the C ABI.
int host_exception() {
    try {
        throw;
    } catch (const std::bad_alloc&) {
        return fail(GRF_ENOMEM, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(GRF_EINVAL, "host exception: %s", e.what());
    } catch (...) {
        return fail(GRF_EINVAL, "unknown host exception");
    }
}
}  // namespace

// NVTX range around one ABI call (visible in Nsight tools and usable as an
// ncu filter; a no-op when no tool is attached).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Every host allocation of the library passes here first.  With failures
// injected (grf_debug_inject_alloc_failures) it fails as the allocator would.
void alloc_point() {
    int32_t v = g_inject_alloc.load();
    while (v > 0)
        if (g_inject_alloc.compare_exchange_weak(v, v - 1)) throw std::bad_alloc();
}

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int set_error(int code, const char* message) { return fail(code, "%s", message); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ---------------------------------------------------------------------------
namespace {
struct Block4 {
    uint32_t w[4];
};

Block4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
    const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = M0 * c0;
        const uint64_t p1 = M1 * c2;
        const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n1 = static_cast<uint32_t>(p1);
        const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ k1;
        const uint32_t n3 = static_cast<uint32_t>(p0);
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    return Block4{{c0, c1, c2, c3}};
}

// Generator stream of one mode: key = seed, counter = (j lo, block, stream, j hi).
class ModeStream {
  public:
    ModeStream(uint64_t seed, uint32_t stream, uint64_t j)
        : k0_(static_cast<uint32_t>(seed)), k1_(static_cast<uint32_t>(seed >> 32)), st_(stream),
          jlo_(static_cast<uint32_t>(j)), jhi_(static_cast<uint32_t>(j >> 32)) {}

    // Two uniforms in (0, 1) from block b: (floor(u64 / 2^12) + 1/2) * 2^-52.
    void uniforms(uint32_t b, double& u0, double& u1) const {
        const Block4 o = philox10(jlo_, b, st_, jhi_, k0_, k1_);
        const uint64_t a = (static_cast<uint64_t>(o.w[1]) << 32) | o.w[0];
        const uint64_t c = (static_cast<uint64_t>(o.w[3]) << 32) | o.w[2];
        const double s = std::ldexp(1.0, -52);
        u0 = (static_cast<double>(a >> 12) + 0.5) * s;
        u1 = (static_cast<double>(c >> 12) + 0.5) * s;
    }
    // Normal number k (Box-Muller of block k / 2; even k cosine, odd k sine).
    double normal(uint32_t k) const {
        double u0, u1;
        uniforms(k / 2, u0, u1);
        const double r = std::sqrt(-2.0 * std::log(u0));
        const double ang = 2.0 * M_PI * u1;
        return (k % 2 == 0) ? r * std::cos(ang) : r * std::sin(ang);
    }

  private:
    uint32_t k0_, k1_, st_, jlo_, jhi_;
};

constexpr int kGammaAttempts = 256;

// Gamma(alpha, 1), alpha >= 1, Marsaglia & Tsang (2000), with the block
// layout of grf_gen_modes.  Returns false if no attempt was accepted.
bool gamma_mt(const ModeStream& g, double alpha, double& out) {
    const double d = alpha - 1.0 / 3.0;
    const double c = 1.0 / std::sqrt(9.0 * d);
    for (int t = 0; t < kGammaAttempts; ++t) {
        const double x = g.normal(2u * (64u + 2u * t));
        double u, unused;
        g.uniforms(65u + 2u * t, u, unused);
        const double v = (1.0 + c * x) * (1.0 + c * x) * (1.0 + c * x);
        if (v <= 0.0) continue;
        if (std::log(u) < 0.5 * x * x + d - d * v + d * std::log(v)) {
            out = d * v;
            return true;
        }
    }
    return false;
}

bool has_rotation(const grf_params* p) {
    for (int k = 0; k < 9; ++k)
        if (p->rot[k] != 0.0) return true;
    return false;
}

// Sec. 4.1 reparameterisation of one mode from its standardised draws:
// A = sigma rho, u = kappa / (2 pi l) per axis, a = R^T u with an axis
// transform, then every periodic axis rounded to a multiple of 1/L_c.
void reparam_one(const grf_params* p, bool rotated, double sigma, const double* kappa, double rho,
                 double* amp, double* a_out) {
    const int d = p->dim;
    *amp = sigma * rho;
    double u[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < d; ++c) u[c] = kappa[c] / (2.0 * M_PI * p->ell[c]);
    for (int c = 0; c < d; ++c) {
        double a = u[c];
        if (rotated) {  // a = R^T u
            a = 0.0;
            for (int k = 0; k < d; ++k) a += p->rot[k * 3 + c] * u[k];
        }
        const double L = p->period[c];
        if (L > 0.0) a = std::floor(a * L + 0.5) / L;  // periodic axis: multiple of 1/L
        a_out[c] = a;
    }
}

int check_params(const grf_params* p) {
    if (!p) return fail(GRF_EINVAL, "params is NULL");
    if (p->family < GRF_GAUSSIAN || p->family > GRF_MATERN)
        return fail(GRF_EINVAL, "unknown covariance family %d", p->family);
    if (p->dim < 1 || p->dim > 3) return fail(GRF_EINVAL, "dim must be 1, 2 or 3 (got %d)", p->dim);
    if (!(p->sigma2 > 0.0) || !std::isfinite(p->sigma2))
        return fail(GRF_EINVAL, "sigma2 must be finite and > 0");
    if (!std::isfinite(p->mean)) return fail(GRF_EINVAL, "mean must be finite");
    for (int c = 0; c < p->dim; ++c)
        if (!(p->ell[c] > 0.0) || !std::isfinite(p->ell[c]))
            return fail(GRF_EINVAL, "ell[%d] must be finite and > 0", c);
    if (p->family == GRF_MATERN && (!(p->nu > 0.0) || !std::isfinite(p->nu)))
        return fail(GRF_EINVAL, "Matern nu must be finite and > 0");
    if (p->n_modes < 1 || p->n_modes > GRF_MAX_MODES)
        return fail(GRF_EINVAL, "n_modes must be in [1, %d]", GRF_MAX_MODES);
    if (p->reserved != 0) return fail(GRF_EINVAL, "reserved field must be 0");
    for (int c = 0; c < 3; ++c)
        if (!(p->period[c] >= 0.0) || !std::isfinite(p->period[c]))
            return fail(GRF_EINVAL, "period[%d] must be finite and >= 0", c);
    if (has_rotation(p)) {
        // any invertible transform of the axes (a rotation, or a general matrix):
        // finite entries and |det| not negligible against the row norms
        const int d = p->dim;
        double m[3][3], rn = 1.0;
        for (int i = 0; i < d; ++i) {
            double r2 = 0.0;
            for (int k = 0; k < d; ++k) {
                m[i][k] = p->rot[i * 3 + k];
                if (!std::isfinite(m[i][k])) return fail(GRF_EINVAL, "rot has a non-finite entry");
                r2 += m[i][k] * m[i][k];
            }
            rn *= std::sqrt(r2);
        }
        double det = m[0][0];
        if (d == 2) det = m[0][0] * m[1][1] - m[0][1] * m[1][0];
        if (d == 3)
            det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                  m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                  m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
        if (!(std::fabs(det) > 1e-12 * rn))
            return fail(GRF_EINVAL, "rot: the leading %dx%d block must be invertible", d, d);
    }
    return GRF_OK;
}

// ---------------------------------------------------------------------------
// Plan registry: host copy of each plan's segment table, keyed by the plan's
// device address (set by grf_plan_cells).
// ---------------------------------------------------------------------------
struct PlanMeta {
    int32_t dim;
    std::vector<int64_t> offsets;
    PlanLayout layout;
    // Cartesian-grid check (single segment, 2-D / 3-D): 0 = not a grid,
    // 1 = pending (its result lands in g_slots[slot] once `ev` completes),
    // 2 = grid of gn[0] x gn[1] x gn[2] cells.
    int32_t grid_state = 0;
    int32_t gn[3] = {0, 0, 0};
    uint64_t tag = 0;
    int32_t slot = -1;
    cudaEvent_t ev = nullptr;
};
std::mutex g_reg_mu;

// Set on the prefetcher's worker threads: each draws whole realisations on
// its own thread, so grf_gen_modes does not start threads of its own there
// (the workers already keep the host cores busy).
thread_local bool t_serial_draw = false;
std::unordered_map<const void*, PlanMeta> g_plans;

// Pinned ring that receives the grid checks of new plans (device -> host
// copies ordered after the planning kernels); a slot reused before its plan
// was first read is recognised by the tag and treated as "not a grid".
constexpr int kGridSlots = 1024;
GridCheck* g_slots = nullptr;
int g_next_slot = 0;
std::atomic<uint64_t> g_next_tag{1};
std::atomic<int32_t> g_grid_enabled{1};  // grf_debug_grid_path: 0 off, 1 auto, 2 always
std::atomic<int32_t> g_grid_fold{4};     // chunks of 32 modes per fold interval

void drop_plan_event(PlanMeta& m) {
    if (m.ev) cudaEventDestroy(m.ev);
    m.ev = nullptr;
}

// Grid path for a grid plan: with the setting on (1, the default, or 2) every
// Cartesian grid takes it -- grids of few tiles split their modes over more
// CTAs and were measured as fast as or faster than the CUDA-core kernels
// (64^2 x 1000 equal, 896 x 128 x 4096 2.5x).
bool use_grid_path(const GridGeom& gg) {
    (void)gg;
    return g_grid_enabled.load() != 0;
}

// The grid path's workspace (tables and partials) grows with the grid's axes
// times N; beyond max(1 GB, 64 B per cell) -- N far above the cell count,
// where the CUDA-core kernels need no tables -- it is not offered.
bool grid_ws_ok(size_t bytes, const GridGeom& gg) {
    const double cells = static_cast<double>(gg.nx) * gg.ny * gg.nz;
    return static_cast<double>(bytes) <= std::max(double(1u << 30), 64.0 * cells);
}

// The grid shape of `plan` (single segment), resolving a pending check by
// waiting for the plan's own event (the planning kernels only).  Returns
// false when the cells are not a Cartesian grid in x-fastest order.
bool plan_grid(const void* plan, GridGeom* gg) {
    PlanMeta m;
    {
        std::lock_guard<std::mutex> lk(g_reg_mu);
        auto it = g_plans.find(plan);
        if (it == g_plans.end()) return false;
        m.grid_state = it->second.grid_state;
        m.ev = it->second.ev;
        m.slot = it->second.slot;
        m.tag = it->second.tag;
        m.dim = it->second.dim;
        m.layout = it->second.layout;
        m.offsets = it->second.offsets;
        for (int c = 0; c < 3; ++c) m.gn[c] = it->second.gn[c];
    }
    if (m.grid_state == 0) return false;
    if (m.grid_state == 1) {
        int32_t st = 0, gn[3] = {0, 0, 0};
        if (cudaEventSynchronize(m.ev) == cudaSuccess) {
            GridCheck c;
            {
                std::lock_guard<std::mutex> lk(g_reg_mu);
                c = g_slots[m.slot];
            }
            const int64_t n = m.offsets.back();
            const int64_t nx = static_cast<int64_t>(c.c1);
            const int64_t nxy = m.dim > 2 ? static_cast<int64_t>(c.c2) : n;
            if (c.tag == m.tag && c.bad == 0 && nx >= 1 && nxy >= nx && nxy % nx == 0 && n % nxy == 0) {
                const int64_t ny = nxy / nx, nz = n / nxy;
                if (ny >= 2 && nx + ny + nz <= n && nx <= INT32_MAX) {
                    st = 2;
                    gn[0] = static_cast<int32_t>(nx);
                    gn[1] = static_cast<int32_t>(ny);
                    gn[2] = static_cast<int32_t>(nz);
                }
            }
        }
        std::lock_guard<std::mutex> lk(g_reg_mu);
        auto it = g_plans.find(plan);
        if (it != g_plans.end() && it->second.tag == m.tag) {
            it->second.grid_state = st;
            for (int c = 0; c < 3; ++c) it->second.gn[c] = gn[c];
            drop_plan_event(it->second);
        }
        m.grid_state = st;
        for (int c = 0; c < 3; ++c) m.gn[c] = gn[c];
    }
    if (m.grid_state != 2) return false;
    const float* axes = reinterpret_cast<const float*>(static_cast<const unsigned char*>(plan) + m.layout.off_keys_in);
    gg->nx = m.gn[0];
    gg->ny = m.gn[1];
    gg->nz = m.gn[2];
    gg->X = axes;
    gg->Y = axes + m.gn[0];
    gg->Z = axes + m.gn[0] + m.gn[1];
    return true;
}

bool lookup_plan(const void* plan, PlanMeta& out) {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    auto it = g_plans.find(plan);
    if (it == g_plans.end()) return false;
    alloc_point();
    out = it->second;
    return true;
}

struct BatchMeta {
    BatchHeader hdr;
    int32_t plan_dim;
};
std::unordered_map<const void*, BatchMeta> g_batches;
std::unordered_map<std::string, std::pair<int32_t, float>> g_tuned;  // batch autotuner cache

MapDev make_map(const grf_map* m, const grf_outputs* out, double mean, double sigma) {
    MapDev d{};
    d.bits = m ? m->bits : 0;
    d.n_thr = m ? m->n_thresholds : 0;
    for (int t = 0; t < GRF_MAX_THRESHOLDS; ++t) d.thr[t] = m ? m->thresholds[t] : 0.f;
    for (int t = 0; t <= GRF_MAX_THRESHOLDS; ++t) d.values[t] = m ? m->values[t] : 0.f;
    d.k_ref = m ? m->k_ref : 1.f;
    d.phi0 = m ? m->phi0 : 0.f;
    d.phi1 = m ? m->phi1 : 0.f;
    d.phi_min = m ? m->phi_min : 0.f;
    d.phi_max = m ? m->phi_max : 0.f;
    d.mu = static_cast<float>(mean);
    d.sigma_inv = static_cast<float>(1.0 / sigma);
    d.Y = out ? out->Y : nullptr;
    d.K = out ? out->K : nullptr;
    d.F = out ? out->facies : nullptr;
    d.P = out ? out->prop : nullptr;
    return d;
}

// Output pointers are required only when there are cells to write (n > 0).
int check_map(const grf_map* m, const grf_outputs* out, int64_t n) {
    if (!m) return fail(GRF_EINVAL, "map is NULL");
    if (!out) return fail(GRF_EINVAL, "outputs is NULL");
    const int known = GRF_MAP_Y | GRF_MAP_LOGNORMAL | GRF_MAP_FACIES | GRF_MAP_VALUES | GRF_MAP_POROSITY;
    if (m->bits & ~known) return fail(GRF_EINVAL, "unknown map bits 0x%x", m->bits);
    if ((m->bits & GRF_MAP_VALUES) && (m->bits & GRF_MAP_POROSITY))
        return fail(GRF_EINVAL, "VALUES and POROSITY share the prop output");
    if (m->n_thresholds < 0 || m->n_thresholds > GRF_MAX_THRESHOLDS)
        return fail(GRF_EINVAL, "n_thresholds must be in [0, %d]", GRF_MAX_THRESHOLDS);
    for (int t = 0; t < m->n_thresholds; ++t) {
        if (!std::isfinite(m->thresholds[t])) return fail(GRF_EINVAL, "threshold %d is not finite", t);
        if (t > 0 && !(m->thresholds[t] > m->thresholds[t - 1]))
            return fail(GRF_EINVAL, "thresholds must be strictly ascending");
    }
    if (n > 0 && (m->bits & GRF_MAP_Y) && !out->Y) return fail(GRF_EINVAL, "Y output is NULL");
    if (n > 0 && (m->bits & GRF_MAP_LOGNORMAL) && !out->K) return fail(GRF_EINVAL, "K output is NULL");
    if (n > 0 && (m->bits & GRF_MAP_FACIES) && !out->facies) return fail(GRF_EINVAL, "facies output is NULL");
    if (n > 0 && (m->bits & (GRF_MAP_VALUES | GRF_MAP_POROSITY)) && !out->prop)
        return fail(GRF_EINVAL, "prop output is NULL");
    if ((m->bits & GRF_MAP_POROSITY) && !(m->phi_min <= m->phi_max))
        return fail(GRF_EINVAL, "phi_min must not exceed phi_max");
    return GRF_OK;
}

}  // namespace
}  // namespace grf

using namespace grf;

extern "C" {

const char* grf_last_error(void) { return g_last_error.c_str(); }

const char* grf_version(void) { return "grf-gb300 1.0"; }

int64_t grf_launch_count(void) { return g_launches.load(); }

int grf_release(const void* buffer) {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    auto it = g_plans.find(buffer);
    if (it != g_plans.end()) drop_plan_event(it->second);
    g_plans.erase(buffer);
    g_batches.erase(buffer);
    return GRF_OK;
}

int grf_debug_inject_alloc_failures(int32_t n) {
    if (n < 0) return fail(GRF_EINVAL, "n must be >= 0");
    g_inject_alloc.store(n);
    return GRF_OK;
}

// ---------------------------------------------------------------------------
// S1: modes
// ---------------------------------------------------------------------------
int grf_gen_modes(const grf_params* p, grf_modes* out) try {
    TraceRange trace_("grf_gen_modes");
    int rc = check_params(p);
    if (rc) return rc;
    if (!out) return fail(GRF_EINVAL, "modes output is NULL");
    if (out->n != p->n_modes || out->dim != p->dim)
        return fail(GRF_EINVAL, "modes arrays sized for n=%lld dim=%d, params say n=%lld dim=%d",
                    (long long)out->n, out->dim, (long long)p->n_modes, p->dim);
    if (!out->kappa || !out->rho || !out->psi || !out->a || !out->amp)
        return fail(GRF_EINVAL, "a modes array is NULL");
    const int64_t N = p->n_modes;
    const int d = p->dim;
    const double sigma = std::sqrt(p->sigma2);
    const double nu = p->family == GRF_EXPONENTIAL ? 0.5 : p->nu;
    const double dof = 2.0 * nu;
    const bool sum_sq = (p->family != GRF_GAUSSIAN) && dof == std::round(dof) && dof >= 1.0 && dof <= 32.0;
    const bool rotated = has_rotation(p);
    // Modes are independent draws: ranges of j run on host threads.  A worker
    // records the first mode whose gamma sampler failed (errors are reported
    // by the calling thread).
    auto draw_range = [&](int64_t j0, int64_t j1, int64_t* bad) {
        for (int64_t j = j0; j < j1; ++j) {
            const ModeStream g(p->seed, p->stream, static_cast<uint64_t>(j));
            const double W = g.normal(0);
            const double Wp = g.normal(1);
            double z[3];
            for (int c = 0; c < d; ++c) z[c] = g.normal(2u + c);
            double scale;
            if (p->family == GRF_GAUSSIAN) {
                scale = std::sqrt(0.5 * M_PI);
            } else {
                double w = 0.0;
                if (sum_sq) {
                    const int m = static_cast<int>(dof);
                    for (int i = 0; i < m; ++i) {
                        const double v = g.normal(static_cast<uint32_t>(2 + d + i));
                        w += v * v;
                    }
                } else {
                    double G;
                    const double alpha = nu >= 1.0 ? nu : nu + 1.0;
                    if (!gamma_mt(g, alpha, G)) {
                        *bad = j;
                        return;
                    }
                    if (nu < 1.0) {
                        double ub, unused;
                        g.uniforms(63u, ub, unused);
                        G *= std::pow(ub, 1.0 / nu);
                    }
                    w = 2.0 * G;
                }
                scale = std::sqrt(dof / w);
            }
            const double rho = std::sqrt((W * W + Wp * Wp) / static_cast<double>(N));
            out->rho[j] = rho;
            out->psi[j] = -std::atan2(Wp, W) / (2.0 * M_PI);
            for (int c = 0; c < d; ++c) out->kappa[j * d + c] = z[c] * scale;
            reparam_one(p, rotated, sigma, out->kappa + j * d, rho, out->amp + j, out->a + j * d);
        }
    };
    constexpr int64_t kModesPerThread = 1024;
    const int64_t hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t nt = t_serial_draw ? 1 : std::min<int64_t>(hw, (N + kModesPerThread - 1) / kModesPerThread);
    alloc_point();
    std::vector<int64_t> bad(static_cast<size_t>(nt), -1);
    if (nt <= 1) {
        draw_range(0, N, &bad[0]);
    } else {
        std::vector<std::thread> pool;
        pool.reserve(static_cast<size_t>(nt));
        try {
            for (int64_t t = 0; t < nt; ++t)
                pool.emplace_back(draw_range, N * t / nt, N * (t + 1) / nt, &bad[static_cast<size_t>(t)]);
        } catch (...) {
            for (auto& th : pool) th.join();  // never destroy a joinable thread
            throw;
        }
        for (auto& th : pool) th.join();
    }
    for (int64_t b : bad)
        if (b >= 0) return fail(GRF_EINVAL, "gamma sampler did not accept for mode %lld", (long long)b);
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_reparam_modes(const grf_params* p, grf_modes* m) try {
    TraceRange trace_("grf_reparam_modes");
    int rc = check_params(p);
    if (rc) return rc;
    if (!m) return fail(GRF_EINVAL, "modes is NULL");
    if (m->n != p->n_modes || m->dim != p->dim)
        return fail(GRF_EINVAL, "modes arrays sized for n=%lld dim=%d, params say n=%lld dim=%d",
                    (long long)m->n, m->dim, (long long)p->n_modes, p->dim);
    if (!m->kappa || !m->rho || !m->a || !m->amp) return fail(GRF_EINVAL, "kappa, rho, a or amp is NULL");
    const int64_t N = m->n;
    const int d = m->dim;
    for (int64_t j = 0; j < N; ++j) {
        if (!std::isfinite(m->rho[j])) return fail(GRF_EINVAL, "rho[%lld] is not finite", (long long)j);
        for (int c = 0; c < d; ++c)
            if (!std::isfinite(m->kappa[j * d + c]))
                return fail(GRF_EINVAL, "kappa of mode %lld is not finite", (long long)j);
    }
    const double sigma = std::sqrt(p->sigma2);
    const bool rotated = has_rotation(p);
    for (int64_t j = 0; j < N; ++j) reparam_one(p, rotated, sigma, m->kappa + j * d, m->rho[j], m->amp + j, m->a + j * d);
    return GRF_OK;
} catch (...) {
    return host_exception();
}

// ---------------------------------------------------------------------------
// Device table
// ---------------------------------------------------------------------------
size_t grf_table_bytes(int64_t n_modes) {
    if (n_modes < 1 || n_modes > GRF_MAX_MODES) return 0;
    return static_cast<size_t>(table_layout(n_modes).total);
}

int grf_pack_table(const grf_modes* m, void* host_table, size_t bytes) try {
    TraceRange trace_("grf_pack_table");
    if (!m || !host_table) return fail(GRF_EINVAL, "modes or table is NULL");
    if (m->n < 1 || m->n > GRF_MAX_MODES) return fail(GRF_EINVAL, "n_modes out of range");
    if (m->dim < 1 || m->dim > 3) return fail(GRF_EINVAL, "dim must be 1, 2 or 3");
    if (!m->a || !m->amp || !m->psi) return fail(GRF_EINVAL, "a, amp or psi array is NULL");
    const TableLayout L = table_layout(m->n);
    if (bytes < static_cast<size_t>(L.total))
        return fail(GRF_EWORKSPACE, "table buffer %zu bytes < %lld needed", bytes, (long long)L.total);
    const int64_t N = m->n;
    const int d = m->dim;
    for (int64_t j = 0; j < N; ++j) {
        if (!std::isfinite(m->amp[j]) || !std::isfinite(m->psi[j]))
            return fail(GRF_EINVAL, "mode %lld has a non-finite amplitude or phase", (long long)j);
        for (int c = 0; c < d; ++c) {
            if (!std::isfinite(m->a[j * d + c]) || std::fabs(m->a[j * d + c]) > kMaxFrequency)
                return fail(GRF_EINVAL, "mode %lld has a frequency that is not finite or exceeds 2^30 turns per unit",
                            (long long)j);
            if (m->kappa && !std::isfinite(m->kappa[j * d + c]))
                return fail(GRF_EINVAL, "mode %lld has a non-finite kappa", (long long)j);
        }
    }
    unsigned char* base = static_cast<unsigned char*>(host_table);
    alloc_point();
    std::vector<double> h(N);
    for (int64_t j = 0; j < N; ++j) {
        double s = 0.0;
        for (int c = 0; c < d; ++c) s += std::fabs(m->a[j * d + c]);
        h[j] = s;
    }
    // order by |a|_1 descending, ties by original index: stable LSD radix sort
    // (8-bit digits) of the complemented bit patterns (h >= 0, so the bits
    // order as the values do)
    std::vector<int64_t> ord(N), tmp(N);
    std::vector<uint64_t> kb(N), kt(N);
    for (int64_t j = 0; j < N; ++j) {
        uint64_t u;
        std::memcpy(&u, &h[j], sizeof(u));
        kb[j] = ~u;
        ord[j] = j;
    }
    for (int shift = 0; shift < 64; shift += 8) {
        int64_t count[257] = {0};
        for (int64_t j = 0; j < N; ++j) ++count[((kb[j] >> shift) & 0xFF) + 1];
        for (int q = 0; q < 256; ++q) count[q + 1] += count[q];
        for (int64_t j = 0; j < N; ++j) {
            const int64_t dst = count[(kb[j] >> shift) & 0xFF]++;
            kt[dst] = kb[j];
            tmp[dst] = ord[j];
        }
        kb.swap(kt);
        ord.swap(tmp);
    }
    std::memset(base, 0, static_cast<size_t>(L.total));

    TableHeader hd{};
    hd.magic = kTableMagic;
    hd.n_modes = static_cast<int32_t>(N);
    hd.n_pad = static_cast<int32_t>(L.n_pad);
    hd.dim = d;
    hd.tau = 1.0f;
    hd.n_buckets = kBuckets;
    hd.bucket_bias = kBucketBias;
    hd.off_hot = L.off_hot;
    hd.off_cold = L.off_cold;
    hd.off_order = L.off_order;
    hd.off_kpref = L.off_kpref;
    hd.off_kappa = L.off_kappa;
    hd.has_kappa = m->kappa != nullptr ? 1 : 0;
    hd.total_bytes = L.total;
    std::memcpy(base, &hd, sizeof(hd));

    float* hot = reinterpret_cast<float*>(base + L.off_hot);
    float* cold = reinterpret_cast<float*>(base + L.off_cold);
    int32_t* order = reinterpret_cast<int32_t*>(base + L.off_order);
    int32_t* kpref = reinterpret_cast<int32_t*>(base + L.off_kpref);
    double* kap = reinterpret_cast<double*>(base + L.off_kappa);
    float amp_max = 0.0f;
    for (int64_t s = 0; s < L.n_pad; ++s) {
        order[s] = -1;
        if (s >= N) continue;
        const int64_t j = ord[s];
        order[s] = static_cast<int32_t>(j);
        if (m->kappa)
            for (int c = 0; c < d; ++c) kap[s * 3 + c] = m->kappa[j * d + c];
        double a[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < d; ++c) a[c] = m->a[j * d + c];
        for (int c = 0; c < 3; ++c) hot[s * 4 + c] = static_cast<float>(2.0 * M_PI * a[c]);
        // (-A, psi + 1/2) at odd positions: see mode_flipped
        const bool flip = mode_flipped(s);
        hot[s * 4 + 3] = static_cast<float>(flip ? -m->amp[j] : m->amp[j]);
        amp_max = std::max(amp_max, std::fabs(hot[s * 4 + 3]));
        const double psi = flip ? (m->psi[j] <= 0.0 ? m->psi[j] + 0.5 : m->psi[j] - 0.5) : m->psi[j];
        float ah[3], al[3];
        for (int c = 0; c < 3; ++c) {
            ah[c] = static_cast<float>(a[c]);
            al[c] = static_cast<float>(a[c] - static_cast<double>(ah[c]));
        }
        const float ph = static_cast<float>(psi);
        const float pl = static_cast<float>(psi - static_cast<double>(ph));
        float* c0 = cold + s * 8;
        c0[0] = ah[0];
        c0[1] = al[0];
        c0[2] = ah[1];
        c0[3] = al[1];
        c0[4] = ah[2];
        c0[5] = al[2];
        c0[6] = ph;
        c0[7] = pl;
    }
    reinterpret_cast<TableHeader*>(base)->amp_max = amp_max;
    // kpref[b] = #{s : h_s * E_b > 1}, E_b = 2^((b - bias) / 4)
    // (E_b grows with b, so the count only grows: one pass over the sorted modes)
    int64_t k = 0;
    for (int b = 0; b < kBuckets; ++b) {
        const double Eb = std::pow(2.0, (b - kBucketBias) / 4.0);
        while (k < N && h[ord[k]] * Eb > 1.0) ++k;
        kpref[b] = static_cast<int32_t>(k);
    }
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_upload_table(const void* host_table, void* dev_table, size_t bytes, void* stream) try {
    TraceRange trace_("grf_upload_table");
    if (!host_table || !dev_table) return fail(GRF_EINVAL, "table pointer is NULL");
    if (!aligned256(dev_table)) return fail(GRF_EINVAL, "device table must be 256-byte aligned");
    TableHeader hd;
    std::memcpy(&hd, host_table, sizeof(hd));
    if (hd.magic != kTableMagic) return fail(GRF_EINVAL, "host table was not built by grf_pack_table");
    if (bytes < static_cast<size_t>(hd.total_bytes))
        return fail(GRF_EWORKSPACE, "device table %zu bytes < %lld needed", bytes, (long long)hd.total_bytes);
    cudaError_t e = cudaMemcpyAsync(dev_table, host_table, static_cast<size_t>(hd.total_bytes),
                                    cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "table upload");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
size_t grf_plan_bytes(int64_t n_cells, int32_t n_segments) {
    if (n_cells < 0 || n_cells > INT32_MAX || n_segments < 1) return 0;
    return static_cast<size_t>(plan_layout(n_cells, n_segments).total);
}

int grf_plan_cells(int32_t dim, int32_t n_segments, const int64_t* seg_offsets, const float* x,
                   const float* y, const float* z, void* plan, size_t plan_bytes, void* stream) try {
    TraceRange trace_("grf_plan_cells");
    if (dim < 1 || dim > 3) return fail(GRF_EINVAL, "dim must be 1, 2 or 3");
    if (n_segments < 1) return fail(GRF_EINVAL, "n_segments must be >= 1");
    if (!seg_offsets) return fail(GRF_EINVAL, "seg_offsets is NULL");
    if (seg_offsets[0] != 0) return fail(GRF_EINVAL, "seg_offsets[0] must be 0");
    for (int s = 0; s < n_segments; ++s)
        if (seg_offsets[s + 1] < seg_offsets[s]) return fail(GRF_EINVAL, "seg_offsets must be ascending");
    const int64_t n = seg_offsets[n_segments];
    if (n > INT32_MAX) return fail(GRF_EINVAL, "at most 2^31-1 cells per plan");
    if (!plan) return fail(GRF_EINVAL, "plan is NULL");
    if (!aligned256(plan)) return fail(GRF_EINVAL, "plan must be 256-byte aligned");
    if (n > 0 && (!x || (dim > 1 && !y) || (dim > 2 && !z)))
        return fail(GRF_EINVAL, "a coordinate array is NULL");
    const PlanLayout L = plan_layout(n, n_segments);
    if (plan_bytes < static_cast<size_t>(L.total))
        return fail(GRF_EWORKSPACE, "plan buffer %zu bytes < %lld needed", plan_bytes, (long long)L.total);
    PlanMeta meta;
    meta.dim = dim;
    alloc_point();
    meta.offsets.assign(seg_offsets, seg_offsets + n_segments + 1);
    meta.layout = L;
    meta.tag = g_next_tag.fetch_add(1);
    const int err = launch_plan(dim, n_segments, seg_offsets, x, y, z, plan, L, meta.tag, stream);
    if (err != cudaSuccess) return cuda_fail(err, "plan kernels");
    std::lock_guard<std::mutex> lk(g_reg_mu);
    if (n_segments == 1 && dim >= 2 && n >= 4) {
        // the grid check's result, copied to a pinned slot after the planning
        // kernels; read (once) by the first call that needs it
        cudaError_t e = cudaSuccess;
        if (!g_slots) e = cudaHostAlloc(reinterpret_cast<void**>(&g_slots), kGridSlots * sizeof(GridCheck),
                                        cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&meta.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            meta.slot = g_next_slot;
            g_next_slot = (g_next_slot + 1) % kGridSlots;
            cudaStream_t st = static_cast<cudaStream_t>(stream);
            e = cudaMemcpyAsync(&g_slots[meta.slot], &static_cast<PlanHeader*>(plan)->grid, sizeof(GridCheck),
                                cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaEventRecord(meta.ev, st);
        }
        if (e != cudaSuccess) {
            drop_plan_event(meta);
            return cuda_fail(e, "grid check read-back");
        }
        meta.grid_state = 1;
    }
    auto it = g_plans.find(plan);
    if (it != g_plans.end()) drop_plan_event(it->second);
    g_plans[plan] = std::move(meta);
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_read_status(const void* plan, int32_t* status_out, void* stream) try {
    if (!plan || !status_out) return fail(GRF_EINVAL, "NULL argument");
    PlanMeta meta;
    if (!lookup_plan(plan, meta)) return fail(GRF_EINVAL, "unknown plan (not built by grf_plan_cells)");
    const PlanHeader* hdr = static_cast<const PlanHeader*>(plan);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(status_out, &hdr->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

// ---------------------------------------------------------------------------
// Synthesis
// ---------------------------------------------------------------------------
namespace {
int fwd_desc(const void* table, int64_t n_modes, int32_t dim, const void* plan,
             const PlanMeta& meta, int32_t segment, const MapDev& map, FwdDesc& d) {
    if (segment < 0 || segment >= static_cast<int32_t>(meta.offsets.size()) - 1)
        return fail(GRF_EINVAL, "segment %d out of range", segment);
    if (dim > meta.dim) return fail(GRF_EINVAL, "field dim %d exceeds plan dim %d", dim, meta.dim);
    if (!aligned256(table)) return fail(GRF_EINVAL, "device table must be 256-byte aligned");
    const TableLayout TL = table_layout(n_modes);
    const unsigned char* tb = static_cast<const unsigned char*>(table);
    const unsigned char* pb = static_cast<const unsigned char*>(plan);
    const int64_t begin = meta.offsets[segment];
    d.hot = reinterpret_cast<const float4*>(tb + TL.off_hot);
    d.cold = reinterpret_cast<const float4*>(tb + TL.off_cold);
    d.kpref = reinterpret_cast<const int32_t*>(tb + TL.off_kpref);
    d.n_pad = static_cast<int32_t>(TL.n_pad);
    d.dim = dim;  // the field's own dimension: coordinates beyond it do not enter the phase
    d.inv_tau1 = 1.0f / kTauLight;
    d.inv_tau2 = 1.0f / kTauMedium;
    d.xs = reinterpret_cast<const float*>(pb + meta.layout.off_xs) + begin;
    d.ys = reinterpret_cast<const float*>(pb + meta.layout.off_ys) + begin;
    d.zs = reinterpret_cast<const float*>(pb + meta.layout.off_zs) + begin;
    d.perm = reinterpret_cast<const int32_t*>(pb + meta.layout.off_perm) + begin;
    d.perm_base = begin;
    d.n_cells = meta.offsets[segment + 1] - begin;
    d.map = map;
    return GRF_OK;
}
}  // namespace

size_t grf_synth_workspace_bytes(int64_t n_cells) {
    if (n_cells < 0) return 0;
    return synth_workspace_bytes(n_cells);
}

int grf_synth_field(const void* table, const grf_params* p, const void* plan, int32_t segment,
                    const grf_map* map, const grf_outputs* out, void* workspace, size_t ws_bytes,
                    void* stream) try {
    TraceRange trace_("grf_synth_field");
    int rc = check_params(p);
    if (rc) return rc;
    if (!table) return fail(GRF_EINVAL, "table is NULL");
    PlanMeta meta;
    if (!plan || !lookup_plan(plan, meta)) return fail(GRF_EINVAL, "unknown plan (not built by grf_plan_cells)");
    const int32_t n_seg = static_cast<int32_t>(meta.offsets.size()) - 1;
    const int64_t n = segment >= 0 && segment < n_seg ? meta.offsets[segment + 1] - meta.offsets[segment] : 0;
    rc = check_map(map, out, n);
    if (rc) return rc;
    if (map->bits == 0) return fail(GRF_EINVAL, "no output requested");
    FwdDesc d{};
    rc = fwd_desc(table, p->n_modes, p->dim, plan, meta, segment,
                  make_map(map, out, p->mean, std::sqrt(p->sigma2)), d);
    if (rc) return rc;
    int32_t* status = &static_cast<PlanHeader*>(const_cast<void*>(plan))->status;
    if (workspace && !aligned256(workspace)) return fail(GRF_EINVAL, "workspace must be 256-byte aligned");
    // Cartesian grid handed over x-fastest: tensor-core path when the
    // workspace holds its tables
    GridGeom gg{};
    if (n > 0 && workspace && g_grid_enabled.load() != 0 && n_seg == 1 && p->dim == meta.dim &&
        plan_grid(plan, &gg) && use_grid_path(gg) &&
        grid_ws_ok(grid_ws_bytes(gg.nx, gg.ny, gg.nz, table_layout(p->n_modes).n_pad), gg) &&
        ws_bytes >= grid_ws_bytes(gg.nx, gg.ny, gg.nz, table_layout(p->n_modes).n_pad)) {
        const int err = launch_synth_grid(table, p->n_modes, p->dim, gg, d.map, workspace, g_grid_fold.load(), status,
                                          stream);
        if (err != cudaSuccess) return cuda_fail(err, "grid synth kernels");
        return GRF_OK;
    }
    const int err = launch_synth_fwd(d, workspace, workspace ? ws_bytes : 0, status, stream);
    if (err != cudaSuccess) return cuda_fail(err, "synth kernel");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

size_t grf_synth_grid_workspace_bytes(const void* plan, int32_t segment, int64_t n_modes) {
    try {
        if (!plan || segment != 0 || n_modes < 1 || n_modes > GRF_MAX_MODES) return 0;
        GridGeom gg{};
        if (!plan_grid(plan, &gg)) return 0;
        const size_t b = grid_ws_bytes(gg.nx, gg.ny, gg.nz, table_layout(n_modes).n_pad);
        return grid_ws_ok(b, gg) ? b : 0;
    } catch (...) {
        return 0;
    }
}

int grf_plan_grid_shape(const void* plan, int32_t* nx, int32_t* ny, int32_t* nz) try {
    if (!plan || !nx || !ny || !nz) return fail(GRF_EINVAL, "NULL argument");
    PlanMeta meta;
    if (!lookup_plan(plan, meta)) return fail(GRF_EINVAL, "unknown plan (not built by grf_plan_cells)");
    GridGeom gg{};
    const bool g = plan_grid(plan, &gg);
    *nx = g ? gg.nx : 0;
    *ny = g ? gg.ny : 0;
    *nz = g ? gg.nz : 0;
    return GRF_OK;
} catch (...) {
    return host_exception();
}

size_t grf_synth_mismatch_workspace_bytes(int64_t n_cells) {
    if (n_cells < 0) return 0;
    return static_cast<size_t>(align256(mismatch_partials(n_cells) * 8)) + synth_workspace_bytes(n_cells);
}

int grf_synth_mismatch(const void* table, const grf_params* p, const void* plan, int32_t segment,
                       const float* K_target, int64_t n_mean, float* gY, double* loss, float* Y_out,
                       float* K_out, void* workspace, size_t ws_bytes, void* stream) try {
    TraceRange trace_("grf_synth_mismatch");
    int rc = check_params(p);
    if (rc) return rc;
    if (!table) return fail(GRF_EINVAL, "table is NULL");
    PlanMeta meta;
    if (!plan || !lookup_plan(plan, meta)) return fail(GRF_EINVAL, "unknown plan (not built by grf_plan_cells)");
    const int32_t n_seg = static_cast<int32_t>(meta.offsets.size()) - 1;
    if (segment < 0 || segment >= n_seg) return fail(GRF_EINVAL, "segment %d out of range", segment);
    const int64_t n = meta.offsets[segment + 1] - meta.offsets[segment];
    if (n_mean == 0) n_mean = n;
    if (n_mean < n) return fail(GRF_EINVAL, "n_mean (%lld) is smaller than the segment's %lld cells",
                                (long long)n_mean, (long long)n);
    if (n > 0 && (!K_target || !gY)) return fail(GRF_EINVAL, "K_target or gY is NULL");
    if (!loss) return fail(GRF_EINVAL, "loss is NULL");
    if (!workspace) return fail(GRF_EINVAL, "workspace is NULL");
    if (!aligned256(workspace)) return fail(GRF_EINVAL, "workspace must be 256-byte aligned");
    const size_t lbytes = static_cast<size_t>(align256(mismatch_partials(n) * 8));
    if (ws_bytes < lbytes)
        return fail(GRF_EWORKSPACE, "mismatch workspace %zu < %zu bytes", ws_bytes, lbytes);
    grf_map m{};
    m.bits = (Y_out ? GRF_MAP_Y : 0) | (K_out ? GRF_MAP_LOGNORMAL : 0);
    m.k_ref = 1.0f;
    grf_outputs o{};
    o.Y = Y_out;
    o.K = K_out;
    MapDev md = make_map(&m, &o, p->mean, std::sqrt(p->sigma2));
    md.bits |= kMapMismatch;
    md.T = K_target;
    md.G = gY;
    md.lpart = static_cast<double*>(workspace);
    md.loss = loss;
    md.inv_n_mean = n_mean > 0 ? 1.0 / static_cast<double>(n_mean) : 0.0;
    md.g_scale = n_mean > 0 ? 2.0f / static_cast<float>(n_mean) : 0.0f;
    FwdDesc d{};
    rc = fwd_desc(table, p->n_modes, p->dim, plan, meta, segment, md, d);
    if (rc) return rc;
    int32_t* status = &static_cast<PlanHeader*>(const_cast<void*>(plan))->status;
    unsigned char* split_ws = static_cast<unsigned char*>(workspace) + lbytes;
    // Cartesian grid: the tensor-core path when the rest of the workspace
    // holds its tables and the loss partials fit
    GridGeom gg{};
    if (n > 0 && g_grid_enabled.load() != 0 && n_seg == 1 && p->dim == meta.dim && plan_grid(plan, &gg) &&
        use_grid_path(gg) && grid_ws_ok(grid_ws_bytes(gg.nx, gg.ny, gg.nz, table_layout(p->n_modes).n_pad), gg) &&
        ws_bytes - lbytes >= grid_ws_bytes(gg.nx, gg.ny, gg.nz, table_layout(p->n_modes).n_pad) &&
        grid_loss_partials(gg.nx, gg.ny, gg.nz) <= mismatch_partials(n)) {
        const int err = launch_synth_grid(table, p->n_modes, p->dim, gg, d.map, split_ws, g_grid_fold.load(),
                                          status, stream);
        if (err != cudaSuccess) return cuda_fail(err, "grid synth kernels");
        return GRF_OK;
    }
    const int err = launch_synth_fwd(d, split_ws, ws_bytes - lbytes, status, stream);
    if (err != cudaSuccess) return cuda_fail(err, "synth kernel");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_map_property(const grf_map* map, double mean, double sigma, int64_t n, const float* Y,
                     const grf_outputs* out, void* stream) try {
    TraceRange trace_("grf_map_property");
    if (n < 0) return fail(GRF_EINVAL, "n must be >= 0");
    int rc = check_map(map, out, n);
    if (rc) return rc;
    if (n > 0 && !Y) return fail(GRF_EINVAL, "Y is NULL");
    if (!(sigma > 0.0)) return fail(GRF_EINVAL, "sigma must be > 0");
    const int err = launch_map(make_map(map, out, mean, sigma), n, Y, stream);
    if (err != cudaSuccess) return cuda_fail(err, "map kernel");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_map_bitruncated(const grf_bimap* map, int64_t n, const float* Y1, const float* Y2, uint8_t* facies,
                        float* prop, void* stream) try {
    TraceRange trace_("grf_map_bitruncated");
    if (!map) return fail(GRF_EINVAL, "map is NULL");
    if (n < 0) return fail(GRF_EINVAL, "n must be >= 0");
    if (n > 0 && (!Y1 || !Y2 || !facies)) return fail(GRF_EINVAL, "Y1, Y2 or facies is NULL");
    if (map->n_t < 0 || map->n_t > GRF_MAX_THRESHOLDS || map->n_s < 0 || map->n_s > GRF_MAX_THRESHOLDS)
        return fail(GRF_EINVAL, "threshold counts must be in [0, %d]", GRF_MAX_THRESHOLDS);
    for (int q = 0; q < map->n_t; ++q)
        if (!std::isfinite(map->t[q]) || (q > 0 && !(map->t[q] > map->t[q - 1])))
            return fail(GRF_EINVAL, "t must be finite and strictly ascending");
    for (int q = 0; q < map->n_s; ++q)
        if (!std::isfinite(map->s[q]) || (q > 0 && !(map->s[q] > map->s[q - 1])))
            return fail(GRF_EINVAL, "s must be finite and strictly ascending");
    const int err = launch_bimap(*map, n, Y1, Y2, facies, prop, stream);
    if (err != cudaSuccess) return cuda_fail(err, "bitruncated map kernel");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

// ---------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------
size_t grf_backward_workspace_bytes(int64_t n_cells, int64_t n_modes, int32_t dim) {
    if (n_modes < 1 || n_modes > GRF_MAX_MODES || dim < 1 || dim > 3 || n_cells < 0) return 0;
    return bwd_workspace_bytes(n_cells, n_modes, dim);
}

size_t grf_backward_grid_workspace_bytes(const void* plan, int32_t segment, int64_t n_modes) {
    try {
        if (!plan || segment != 0 || n_modes < 1 || n_modes > GRF_MAX_MODES) return 0;
        GridGeom gg{};
        if (!plan_grid(plan, &gg)) return 0;
        const size_t b = bwd_grid_ws_bytes(gg.nx, gg.ny, gg.nz, table_layout(n_modes).n_pad);
        return grid_ws_ok(b, gg) ? b : 0;
    } catch (...) {
        return 0;
    }
}

int grf_synth_backward(const void* table, const grf_params* p, const void* plan, int32_t segment,
                       const float* gY, const grf_grads* g, void* workspace, size_t ws_bytes,
                       void* stream) try {
    TraceRange trace_("grf_synth_backward");
    int rc = check_params(p);
    if (rc) return rc;
    if (!table || !g || !g->dA || !g->dpsi || !g->da || !g->dmu || !g->dsigma || !g->dell)
        return fail(GRF_EINVAL, "table or a gradient output is NULL");
    PlanMeta meta;
    if (!plan || !lookup_plan(plan, meta)) return fail(GRF_EINVAL, "unknown plan (not built by grf_plan_cells)");
    if (p->dim != meta.dim) return fail(GRF_EINVAL, "params dim %d != plan dim %d", p->dim, meta.dim);
    if (segment < 0 || segment >= static_cast<int32_t>(meta.offsets.size()) - 1)
        return fail(GRF_EINVAL, "segment %d out of range", segment);
    const int64_t begin = meta.offsets[segment];
    const int64_t n = meta.offsets[segment + 1] - begin;
    if (n > 0 && !gY) return fail(GRF_EINVAL, "gY is NULL");
    if (!workspace) return fail(GRF_EINVAL, "workspace is NULL");
    if (!aligned256(workspace)) return fail(GRF_EINVAL, "workspace must be 256-byte aligned");
    if (!aligned256(table)) return fail(GRF_EINVAL, "device table must be 256-byte aligned");
    const unsigned char* pb = static_cast<const unsigned char*>(plan);
    int32_t* status = &static_cast<PlanHeader*>(const_cast<void*>(plan))->status;
    double rot[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (has_rotation(p))
        for (int k = 0; k < 9; ++k) rot[k] = p->rot[k];
    int32_t periodic = 0;
    for (int c = 0; c < p->dim; ++c)
        if (p->period[c] > 0.0) periodic |= 1 << c;
    // Cartesian grid handed over x-fastest: the tensor-core adjoint when the
    // workspace holds its tables
    GridGeom gg{};
    if (n > 0 && g_grid_enabled.load() != 0 && meta.offsets.size() == 2 && p->dim >= 2 && plan_grid(plan, &gg) &&
        use_grid_path(gg) && grid_ws_ok(bwd_grid_ws_bytes(gg.nx, gg.ny, gg.nz, table_layout(p->n_modes).n_pad), gg) &&
        ws_bytes >= bwd_grid_ws_bytes(gg.nx, gg.ny, gg.nz, table_layout(p->n_modes).n_pad)) {
        const int err = launch_synth_bwd_grid(table, p->n_modes, p->dim, gg, gY, std::sqrt(p->sigma2), p->ell, rot,
                                              periodic, *g, workspace, status, stream);
        if (err != cudaSuccess) return cuda_fail(err, "grid backward kernels");
        return GRF_OK;
    }
    const size_t need = bwd_workspace_bytes(n, p->n_modes, p->dim);
    if (ws_bytes < need) return fail(GRF_EWORKSPACE, "backward workspace %zu < %zu bytes", ws_bytes, need);
    const int err = launch_synth_bwd(
        table, p->n_modes, p->dim, std::sqrt(p->sigma2), p->ell, rot, periodic,
        reinterpret_cast<const float*>(pb + meta.layout.off_xs) + begin,
        reinterpret_cast<const float*>(pb + meta.layout.off_ys) + begin,
        reinterpret_cast<const float*>(pb + meta.layout.off_zs) + begin,
        reinterpret_cast<const int32_t*>(pb + meta.layout.off_perm) + begin, begin, n, gY, *g,
        workspace, status, stream);
    if (err != cudaSuccess) return cuda_fail(err, "backward kernels");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

size_t grf_mismatch_workspace_bytes(int64_t n) {
    if (n < 0) return 0;
    return mismatch_workspace_bytes(n);
}

int grf_mismatch_grad(int64_t n, const float* K, const float* K_target, float* gY, double* loss,
                      void* workspace, size_t ws_bytes, void* stream) try {
    TraceRange trace_("grf_mismatch_grad");
    if (n < 0) return fail(GRF_EINVAL, "n must be >= 0");
    if (n > 0 && (!K || !K_target || !gY)) return fail(GRF_EINVAL, "K, K_target or gY is NULL");
    if (!loss || !workspace) return fail(GRF_EINVAL, "loss or workspace is NULL");
    const size_t need = mismatch_workspace_bytes(n);
    if (ws_bytes < need) return fail(GRF_EWORKSPACE, "mismatch workspace %zu < %zu bytes", ws_bytes, need);
    const int err = launch_mismatch(n, K, K_target, gY, loss, workspace, stream);
    if (err != cudaSuccess) return cuda_fail(err, "mismatch kernels");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

// ---------------------------------------------------------------------------
// Batched ensembles
// ---------------------------------------------------------------------------
size_t grf_batch_workspace_bytes(int32_t n_items, int64_t n_cells) {
    if (n_items < 1 || n_cells < 0) return 0;
    const int64_t min_tile = 128;
    const int64_t max_work = n_cells / min_tile + n_items;
    return static_cast<size_t>(256 + align256(int64_t(n_items) * int64_t(sizeof(FwdDesc))) +
                               align256(max_work * int64_t(sizeof(WorkItem))) + 256);
}

int grf_batch_prepare(int32_t n_items, const grf_batch_item* items, const void* plan,
                      int32_t tile_cells, void* workspace, size_t ws_bytes, void* host_staging,
                      void* stream) try {
    TraceRange trace_("grf_batch_prepare");
    if (n_items < 1 || !items) return fail(GRF_EINVAL, "no batch items");
    if (!workspace || !host_staging) return fail(GRF_EINVAL, "workspace or staging is NULL");
    if (!aligned256(workspace)) return fail(GRF_EINVAL, "workspace must be 256-byte aligned");
    PlanMeta meta;
    if (!plan || !lookup_plan(plan, meta)) return fail(GRF_EINVAL, "unknown plan (not built by grf_plan_cells)");
    int cfg;
    switch (tile_cells) {
        case 0:
        case 256: cfg = 0; break;
        case 128: cfg = 1; break;
        case 512: cfg = 2; break;
        default: return fail(GRF_EINVAL, "tile_cells must be 0, 128, 256 or 512");
    }
    const int64_t tc = fwd_tile_cells(cfg);
    const size_t need = grf_batch_workspace_bytes(n_items, meta.offsets.back());
    if (ws_bytes < need) return fail(GRF_EWORKSPACE, "batch workspace %zu < %zu bytes", ws_bytes, need);
    BatchHeader h{};
    h.magic = kBatchMagic;
    h.n_items = n_items;
    h.tile_cells = static_cast<int32_t>(tc);
    h.cfg = cfg;
    h.dim_max = meta.dim;
    h.off_desc = 256;
    h.off_work = h.off_desc + align256(int64_t(n_items) * int64_t(sizeof(FwdDesc)));
    unsigned char* hs = static_cast<unsigned char*>(host_staging);
    FwdDesc* descs = reinterpret_cast<FwdDesc*>(hs + h.off_desc);
    alloc_point();
    std::vector<int64_t> order(n_items);
    for (int32_t r = 0; r < n_items; ++r) {
        const grf_batch_item& it = items[r];
        if (!it.table) return fail(GRF_EINVAL, "item %d: table is NULL", r);
        if (it.n_modes < 1 || it.n_modes > GRF_MAX_MODES) return fail(GRF_EINVAL, "item %d: n_modes", r);
        if (it.dim < 1 || it.dim > 3) return fail(GRF_EINVAL, "item %d: dim", r);
        if (!(it.sigma > 0.0) || !std::isfinite(it.mean)) return fail(GRF_EINVAL, "item %d: sigma/mean", r);
        const int32_t n_seg = static_cast<int32_t>(meta.offsets.size()) - 1;
        const int64_t n_it = it.segment >= 0 && it.segment < n_seg
                                 ? meta.offsets[it.segment + 1] - meta.offsets[it.segment]
                                 : 0;
        int rc = check_map(&it.map, &it.out, n_it);
        if (rc) return fail(rc, "item %d: %s", r, g_last_error.c_str());
        if (it.map.bits == 0) return fail(GRF_EINVAL, "item %d: no output requested", r);
        FwdDesc d{};
        rc = fwd_desc(it.table, it.n_modes, it.dim, plan, meta, it.segment,
                      make_map(&it.map, &it.out, it.mean, it.sigma), d);
        if (rc) return fail(rc, "item %d: %s", r, g_last_error.c_str());
        std::memcpy(&descs[r], &d, sizeof(FwdDesc));
        order[r] = r;
    }
    // longest-processing-time first: realisations with more modes first
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t u, int64_t v) { return descs[u].n_pad > descs[v].n_pad; });
    WorkItem* work = reinterpret_cast<WorkItem*>(hs + h.off_work);
    int64_t nw = 0;
    const int64_t cap = (static_cast<int64_t>(need) - h.off_work) / int64_t(sizeof(WorkItem));
    for (int64_t q = 0; q < n_items; ++q) {
        const int64_t r = order[q];
        const int64_t tiles = (descs[r].n_cells + tc - 1) / tc;
        for (int64_t t = 0; t < tiles; ++t) {
            if (nw >= cap) return fail(GRF_EWORKSPACE, "work list exceeds workspace");
            work[nw].r = static_cast<int32_t>(r);
            work[nw].t = static_cast<int32_t>(t);
            ++nw;
        }
    }
    h.n_work = static_cast<int32_t>(nw);
    h.off_counter = h.off_work + align256(nw * int64_t(sizeof(WorkItem)));
    h.total_bytes = h.off_counter + 256;
    std::memcpy(hs, &h, sizeof(h));
    cudaError_t e = cudaMemcpyAsync(workspace, host_staging, static_cast<size_t>(h.off_counter),
                                    cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "batch descriptor upload");
    BatchMeta bm{h, meta.dim};
    std::lock_guard<std::mutex> lk(g_reg_mu);
    g_batches[workspace] = bm;
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_batch_autotune(int32_t n_items, const grf_batch_item* items, const void* plan, void* workspace,
                       size_t ws_bytes, void* host_staging, void* stream, int32_t* tile_cells,
                       float* best_ms) try {
    TraceRange trace_("grf_batch_autotune");
    if (!tile_cells || !best_ms) return fail(GRF_EINVAL, "tile_cells or best_ms is NULL");
    if (n_items < 1 || !items) return fail(GRF_EINVAL, "no batch items");
    PlanMeta meta;
    if (!plan || !lookup_plan(plan, meta)) return fail(GRF_EINVAL, "unknown plan (not built by grf_plan_cells)");
    // signature of the batch layout
    double cell_modes = 0.0;
    int64_t cells = 0;
    for (int32_t r = 0; r < n_items; ++r) {
        const int32_t sg = items[r].segment;
        if (sg < 0 || sg >= static_cast<int32_t>(meta.offsets.size()) - 1)
            return fail(GRF_EINVAL, "item %d: segment out of range", r);
        const int64_t c = meta.offsets[sg + 1] - meta.offsets[sg];
        cells += c;
        cell_modes += static_cast<double>(c) * static_cast<double>(items[r].n_modes);
    }
    char key[160];
    std::snprintf(key, sizeof(key), "%d/%lld/%.6e/%d", n_items, (long long)cells, cell_modes, meta.dim);
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_reg_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            *tile_cells = it->second.first;
            *best_ms = it->second.second;
            cached = true;
        }
    }
    // (the registry lock is released before grf_batch_prepare takes it again)
    if (cached)
        return grf_batch_prepare(n_items, items, plan, *tile_cells, workspace, ws_bytes, host_staging, stream);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(GRF_ECUDA, "event creation failed");
    const int32_t candidates[3] = {256, 512, 128};
    int32_t best = 0;
    float best_t = 0.f;
    int rc = GRF_OK;
    for (int32_t tc : candidates) {
        rc = grf_batch_prepare(n_items, items, plan, tc, workspace, ws_bytes, host_staging, stream);
        if (rc) break;
        rc = grf_batch_launch(workspace, stream);  // warm-up
        if (rc) break;
        cudaEventRecord(e0, st);
        rc = grf_batch_launch(workspace, stream);
        if (rc) break;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = fail(GRF_ECUDA, "autotune timing failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best == 0 || ms < best_t) {
            best = tc;
            best_t = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_reg_mu);
        g_tuned[key] = std::make_pair(best, best_t);
    }
    *tile_cells = best;
    *best_ms = best_t;
    return grf_batch_prepare(n_items, items, plan, best, workspace, ws_bytes, host_staging, stream);
} catch (...) {
    return host_exception();
}

int grf_batch_launch(void* workspace, void* stream) try {
    TraceRange trace_("grf_batch_launch");
    BatchMeta bm;
    {
        std::lock_guard<std::mutex> lk(g_reg_mu);
        auto it = g_batches.find(workspace);
        if (it == g_batches.end()) return fail(GRF_EINVAL, "workspace was not prepared by grf_batch_prepare");
        bm = it->second;
    }
    unsigned char* base = static_cast<unsigned char*>(workspace);
    int32_t* counter = reinterpret_cast<int32_t*>(base + bm.hdr.off_counter);
    int32_t* status = counter + 1;
    const int err = launch_synth_batched(workspace, bm.hdr, status, counter, stream);
    if (err != cudaSuccess) return cuda_fail(err, "batched kernel");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

// ---------------------------------------------------------------------------
// Mode prefetcher: realisations drawn and packed ahead of use on host threads
// ---------------------------------------------------------------------------
}  // extern "C"

struct grf_prefetch {
    enum State { kFree, kDrawing, kReady, kUploaded };
    grf_params p{};
    int32_t depth = 0;
    int device = 0;
    size_t table_bytes = 0;
    std::vector<void*> slots;        // caller's pinned host staging buffers
    std::vector<cudaEvent_t> events; // upload of each slot, recorded by grf_prefetch_next
    std::vector<State> state;
    std::vector<int64_t> index;      // realisation a ready slot holds
    int64_t next_draw = 0;           // next realisation a worker claims
    int64_t next_use = 0;            // next realisation grf_prefetch_next hands out
    bool stop = false;
    int error = GRF_OK;
    std::string error_msg;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::thread> workers;

    void fail_with(int code, const std::string& msg) {
        std::lock_guard<std::mutex> lk(mu);
        if (error == GRF_OK) {
            error = code;
            error_msg = msg;
        }
        cv.notify_all();
    }

    // Worker: claim the next realisation k once slot k % depth is no longer
    // needed (realisation k - depth handed out and its upload finished), draw
    // its modes with seed p.seed + k, pack them into the slot, mark it ready.
    void work() {
        if (cudaSetDevice(device) != cudaSuccess) {
            fail_with(GRF_ECUDA, "prefetch worker: cudaSetDevice failed");
            return;
        }
        t_serial_draw = true;
        const int64_t N = p.n_modes;
        const int d = p.dim;
        std::vector<double> kappa, rho, psi, a, amp;
        try {
            kappa.resize(N * d);
            rho.resize(N);
            psi.resize(N);
            a.resize(N * d);
            amp.resize(N);
        } catch (const std::bad_alloc&) {
            fail_with(GRF_ENOMEM, "prefetch worker: host allocation failed");
            return;
        }
        grf_modes m{};
        m.n = N;
        m.dim = d;
        m.kappa = kappa.data();
        m.rho = rho.data();
        m.psi = psi.data();
        m.a = a.data();
        m.amp = amp.data();
        for (;;) {
            int64_t k;
            int32_t s;
            bool wait_upload;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return stop || error != GRF_OK || next_draw - next_use < depth; });
                if (stop || error != GRF_OK) return;
                k = next_draw++;
                s = static_cast<int32_t>(k % depth);
                wait_upload = state[s] == kUploaded;
                state[s] = kDrawing;
            }
            if (wait_upload && cudaEventSynchronize(events[s]) != cudaSuccess) {
                fail_with(GRF_ECUDA, "prefetch worker: waiting for a staging slot's upload failed");
                return;
            }
            grf_params pk = p;
            pk.seed = p.seed + static_cast<uint64_t>(k);
            int rc = grf_gen_modes(&pk, &m);
            if (rc == GRF_OK) rc = grf_pack_table(&m, slots[s], table_bytes);
            if (rc != GRF_OK) {
                fail_with(rc, std::string("prefetch worker: ") + grf_last_error());
                return;
            }
            std::lock_guard<std::mutex> lk(mu);
            state[s] = kReady;
            index[s] = k;
            cv.notify_all();
        }
    }
};

extern "C" {

int grf_prefetch_create(const grf_params* p, int32_t depth, int32_t threads, void* const* host_slots,
                        size_t slot_bytes, grf_prefetch** out) try {
    TraceRange trace_("grf_prefetch_create");
    int rc = check_params(p);
    if (rc) return rc;
    if (!out) return fail(GRF_EINVAL, "out is NULL");
    *out = nullptr;
    if (depth < 2 || depth > 64) return fail(GRF_EINVAL, "depth must be in [2, 64]");
    if (threads < 1 || threads > 64) return fail(GRF_EINVAL, "threads must be in [1, 64]");
    if (!host_slots) return fail(GRF_EINVAL, "host_slots is NULL");
    for (int32_t s = 0; s < depth; ++s)
        if (!host_slots[s]) return fail(GRF_EINVAL, "host slot %d is NULL", s);
    const size_t tb = grf_table_bytes(p->n_modes);
    if (slot_bytes < tb) return fail(GRF_EWORKSPACE, "staging slots of %zu bytes < %zu needed", slot_bytes, tb);
    alloc_point();
    std::unique_ptr<grf_prefetch> pf(new grf_prefetch());
    pf->p = *p;
    pf->depth = depth;
    pf->table_bytes = tb;
    if (cudaGetDevice(&pf->device) != cudaSuccess) return fail(GRF_ECUDA, "cudaGetDevice failed");
    pf->slots.assign(host_slots, host_slots + depth);
    pf->state.assign(depth, grf_prefetch::kFree);
    pf->index.assign(depth, -1);
    for (int32_t s = 0; s < depth; ++s) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            for (cudaEvent_t x : pf->events) cudaEventDestroy(x);
            return fail(GRF_ECUDA, "event creation failed");
        }
        pf->events.push_back(e);
    }
    try {
        for (int32_t t = 0; t < threads; ++t) pf->workers.emplace_back(&grf_prefetch::work, pf.get());
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(pf->mu);
            pf->stop = true;
        }
        pf->cv.notify_all();
        for (auto& th : pf->workers) th.join();
        for (cudaEvent_t x : pf->events) cudaEventDestroy(x);
        throw;
    }
    *out = pf.release();
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_prefetch_next(grf_prefetch* pf, void* dev_table, size_t bytes, void* stream, uint64_t* seed_out) try {
    TraceRange trace_("grf_prefetch_next");
    if (!pf || !dev_table) return fail(GRF_EINVAL, "prefetcher or device table is NULL");
    if (!aligned256(dev_table)) return fail(GRF_EINVAL, "device table must be 256-byte aligned");
    if (bytes < pf->table_bytes) return fail(GRF_EWORKSPACE, "device table %zu bytes < %zu needed", bytes,
                                             pf->table_bytes);
    std::unique_lock<std::mutex> lk(pf->mu);
    const int64_t k = pf->next_use;
    const int32_t s = static_cast<int32_t>(k % pf->depth);
    pf->cv.wait(lk, [&] {
        return pf->error != GRF_OK || (pf->state[s] == grf_prefetch::kReady && pf->index[s] == k);
    });
    if (pf->error != GRF_OK) return fail(pf->error, "%s", pf->error_msg.c_str());
    lk.unlock();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(dev_table, pf->slots[s], pf->table_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(pf->events[s], st);
    if (e != cudaSuccess) {
        pf->fail_with(GRF_ECUDA, "prefetch: table upload failed");
        return cuda_fail(e, "prefetch table upload");
    }
    lk.lock();
    pf->state[s] = grf_prefetch::kUploaded;
    pf->next_use = k + 1;
    pf->cv.notify_all();
    if (seed_out) *seed_out = pf->p.seed + static_cast<uint64_t>(k);
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_prefetch_destroy(grf_prefetch* pf) try {
    if (!pf) return GRF_OK;
    {
        std::lock_guard<std::mutex> lk(pf->mu);
        pf->stop = true;
    }
    pf->cv.notify_all();
    for (auto& th : pf->workers) th.join();
    int rc = GRF_OK;
    for (int32_t s = 0; s < pf->depth; ++s) {
        // the caller may free the staging buffers once this returns
        if (pf->state[s] == grf_prefetch::kUploaded && cudaEventSynchronize(pf->events[s]) != cudaSuccess)
            rc = fail(GRF_ECUDA, "waiting for an upload from a staging slot failed");
        cudaEventDestroy(pf->events[s]);
    }
    delete pf;
    return rc;
} catch (...) {
    return host_exception();
}

// ---------------------------------------------------------------------------
// Measurement helpers
// ---------------------------------------------------------------------------
int grf_device_info(int32_t* sm_count, int32_t* sm_clock_khz) try {
    if (!sm_count || !sm_clock_khz) return fail(GRF_EINVAL, "NULL argument");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(sm_clock_khz, cudaDevAttrClockRate, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device attributes");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_selftest_wait(int32_t limit_us, int32_t* status_dev, void* stream) try {
    if (limit_us < 1 || limit_us > 2000000) return fail(GRF_EINVAL, "limit_us must be in [1, 2000000]");
    if (!status_dev) return fail(GRF_EINVAL, "status_dev is NULL");
    int err = launch_selftest_wait(static_cast<uint64_t>(limit_us) * 1000ull, status_dev, stream);
    if (err != cudaSuccess) return cuda_fail(err, "self-test kernel");
    int32_t st = -1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(&st, status_dev, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "self-test status read");
    if (st == 2) return fail(GRF_ETIMEOUT, "bounded device wait expired after %d us (expected)", limit_us);
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_checked_build(void) { return GRF_CHECKED ? 1 : 0; }

int grf_take_index_faults(int64_t* count_out) try {
    if (!count_out) return fail(GRF_EINVAL, "count_out is NULL");
    *count_out = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before reading the index-fault counters");
    unsigned long long total = 0ull;
    for (unsigned long long v : {take_index_faults_fwd(), take_index_faults_bwd(), take_index_faults_plan()}) {
        if (v == ~0ull) return fail(GRF_ECUDA, "index-fault counter not readable");
        total += v;
    }
    *count_out = static_cast<int64_t>(total);
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_take_path_counts(int64_t* general_warps, int64_t* lattice_warps) try {
    if (!general_warps || !lattice_warps) return fail(GRF_EINVAL, "NULL argument");
    *general_warps = 0;
    *lattice_warps = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before reading the path counters");
    unsigned long long g = 0ull, l = 0ull;
    e = static_cast<cudaError_t>(take_path_counts(&g, &l));
    if (e != cudaSuccess) return cuda_fail(e, "path counters");
    *general_warps = static_cast<int64_t>(g);
    *lattice_warps = static_cast<int64_t>(l);
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_take_adjoint_path_counts(int64_t* general_tiles, int64_t* lattice_tiles) try {
    if (!general_tiles || !lattice_tiles) return fail(GRF_EINVAL, "NULL argument");
    *general_tiles = 0;
    *lattice_tiles = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before reading the path counters");
    unsigned long long g = 0ull, l = 0ull;
    e = static_cast<cudaError_t>(take_bwd_path_counts(&g, &l));
    if (e != cudaSuccess) return cuda_fail(e, "adjoint path counters");
    *general_tiles = static_cast<int64_t>(g);
    *lattice_tiles = static_cast<int64_t>(l);
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_take_grid_tiles(int64_t* tiles) try {
    if (!tiles) return fail(GRF_EINVAL, "NULL argument");
    *tiles = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before reading the grid tile counter");
    unsigned long long v = 0ull;
    e = static_cast<cudaError_t>(take_grid_tiles(&v));
    if (e != cudaSuccess) return cuda_fail(e, "grid tile counter");
    *tiles = static_cast<int64_t>(v);
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_take_grid_adjoint_units(int64_t* units) try {
    if (!units) return fail(GRF_EINVAL, "NULL argument");
    *units = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before reading the grid adjoint unit counter");
    unsigned long long v = 0ull;
    e = static_cast<cudaError_t>(take_grid_adj_units(&v));
    if (e != cudaSuccess) return cuda_fail(e, "grid adjoint unit counter");
    *units = static_cast<int64_t>(v);
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_debug_grid_path(int32_t enable, int32_t fold_chunks) {
    if (fold_chunks != 1 && fold_chunks != 2 && fold_chunks != 4 && fold_chunks != 8)
        return fail(GRF_EINVAL, "fold_chunks must be 1, 2, 4 or 8");
    if (enable < 0 || enable > 2) return fail(GRF_EINVAL, "enable must be 0, 1 or 2");
    g_grid_enabled.store(enable);
    g_grid_fold.store(fold_chunks);
    return GRF_OK;
}

int grf_debug_mma_f16(const uint16_t* A, const uint16_t* B, int32_t k_chunks, float* D, int32_t* status_dev,
                      void* stream) try {
    if (!A || !B || !D || !status_dev) return fail(GRF_EINVAL, "NULL argument");
    if (k_chunks < 1 || k_chunks > 4096) return fail(GRF_EINVAL, "k_chunks must be in [1, 4096]");
    const int err = launch_mma_probe(A, B, k_chunks, D, status_dev, stream);
    if (err != cudaSuccess) return cuda_fail(err, "MMA self-test kernel");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

int grf_mufu_probe(int32_t blocks, int32_t iters, float* sink, void* stream) try {
    if (blocks < 1 || iters < 1 || !sink) return fail(GRF_EINVAL, "bad probe arguments");
    const int err = launch_mufu_probe(blocks, iters, sink, stream);
    if (err != cudaSuccess) return cuda_fail(err, "probe kernel");
    return GRF_OK;
} catch (...) {
    return host_exception();
}

}  // extern "C"
