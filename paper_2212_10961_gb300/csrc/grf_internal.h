// Internal layout shared by the host code and the CUDA kernels of the
// spectral Gaussian-random-field library.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include "grf.h"

#ifndef GRF_CHECKED
#define GRF_CHECKED 0  // 1 in the checked build (libgrf_checked.so)
#endif

namespace grf {

// ---------------------------------------------------------------------------
// Device mode table (built on the host by grf_pack_table).
//
// Modes are stored in decreasing order of h_j = sum_c |a_jc| (turns per unit
// length) and padded with zero-amplitude modes to a multiple of kChunk, so the
// chunked loops need no tail.  Sections (byte offsets from the table start,
// all 256-byte aligned):
//   hot  : float4[n_pad]   (2 pi a_x, 2 pi a_y, 2 pi a_z, A)  -- radians/unit
//   cold : float4[2*n_pad] (ah_x, al_x, ah_y, al_y), (ah_z, al_z, psi_h, psi_l)
//          a = ah + al and psi = psi_h + psi_l as FP32 pairs (turns)
//   order: int32[n_pad]    original mode index j (-1 for padding)
//   kpref: int32[kBuckets] kpref[b] = #{j : h_j * 2^((b - bias)/4) > 1}, the
//          length of the prefix of modes whose phase span over a box of
//          half-extent E exceeds tau turns is read at bucket(E / tau)
//   kappa: double[3*n_pad] standardised wave-vector of the mode in the slot
//          (zeros beyond dim and for padding); filled when the modes were
//          packed with their kappa (header has_kappa = 1).  Only the adjoint
//          reads it: the chain rule to l and R needs u = kappa / (2 pi l),
//          which a periodic axis's rounded frequency no longer determines.
// Every mode at an odd sorted position is stored in the equivalent form
// (-A, psi + 1/2): A cos(2 pi (a.x + psi)) = -A cos(2 pi (a.x + psi + 1/2)).
// Half of the terms then evaluate the hardware cosine half a turn away with
// the opposite sign, so a mean offset of its error over the phases cancels
// between the two halves instead of adding up over all N terms (it would
// otherwise grow like c * sum_j A_j ~ sqrt(N)).  Only the adjoint's dA_j
// changes sign with the form (dpsi, da and the chain rule are invariant).
// ---------------------------------------------------------------------------
constexpr int kChunk = 128;          // modes per shared-memory chunk
constexpr int kBuckets = 160;        // extent buckets
constexpr int kBucketBias = 100;     // E_b = 2^((b - kBucketBias) / 4)
constexpr float kTauLight = 8.0f;    // warp-origin path iff h_j * E_warp <= tau1 (turns)
constexpr float kTauMedium = 16.0f;  // lane-origin path iff h_j * E_lane <= tau2 (turns)
constexpr uint32_t kTableMagic = 0x54465247u;  // "GRFT"

// Sorted position s holds its mode in the form (-A, psi + 1/2).
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr bool mode_flipped(int64_t s) { return (s & 1) != 0; }
// Largest |a_c| (turns per unit length) accepted: with |x| < 2^16 the exact
// phase split needs |a x| < 2^46.
constexpr double kMaxFrequency = 1073741824.0;  // 2^30

struct TableHeader {
    uint32_t magic;
    int32_t n_modes;
    int32_t n_pad;
    int32_t dim;
    float tau;
    int32_t n_buckets;
    int32_t bucket_bias;
    int32_t has_kappa;  // 1: the kappa section holds the modes' kappa
    int64_t off_hot;
    int64_t off_cold;
    int64_t off_order;
    int64_t off_kpref;
    int64_t total_bytes;
    int64_t off_kappa;
    float amp_max;      // largest |A_j| as stored (FP32): the grid path's operand scale
    int32_t pad_;
    int64_t reserved[5];
};
static_assert(sizeof(TableHeader) <= 256, "table header must fit in 256 bytes");

inline int64_t align256(int64_t v) { return (v + 255) & ~int64_t(255); }
inline int64_t pad_modes(int64_t n) { return (n + kChunk - 1) / kChunk * kChunk; }

struct TableLayout {
    int64_t n_pad, off_hot, off_cold, off_order, off_kpref, off_kappa, total;
};

inline TableLayout table_layout(int64_t n_modes) {
    TableLayout L;
    L.n_pad = pad_modes(n_modes);
    L.off_hot = 256;
    L.off_cold = L.off_hot + align256(L.n_pad * 16);
    L.off_order = L.off_cold + align256(L.n_pad * 32);
    L.off_kpref = L.off_order + align256(L.n_pad * 4);
    L.off_kappa = L.off_kpref + align256(kBuckets * 4);
    L.total = L.off_kappa + align256(L.n_pad * 24);
    return L;
}

// ---------------------------------------------------------------------------
// Cell plan (device buffer built by grf_plan_cells).
//   header  : PlanHeader (256 B)
//   segs    : SegInfo[n_segments]
//   xs,ys,zs: float[n_cells] sorted coordinates
//   perm    : int32[n_cells] original (plan-global) index of sorted cell i
//   keys_in, keys_out : uint32[n_cells]   (planning scratch)
//   vals_in           : int32[n_cells]    (planning scratch)
//   sort_tmp          : radix-sort temporary storage
// ---------------------------------------------------------------------------
constexpr uint32_t kPlanMagic = 0x4E4C5047u;  // "GPLN"

struct GridCheck {
    unsigned long long c1;  // min {n >= 1 : (y_n, z_n) != (y_0, z_0)}, n_cells if none
    unsigned long long c2;  // min {n >= 1 : z_n != z_0}, n_cells if none (3-D)
    int32_t bad;            // some cell is not at (X_i, Y_k, Z_l) of its index
    int32_t pad_;
    uint64_t tag;           // host-assigned plan number
};
constexpr int kMortonBits = 10;                // quantised coordinate bits per axis

struct PlanHeader {
    uint32_t magic;
    int32_t status;       // device-side error bits
    int32_t dim;
    int32_t n_segments;
    int64_t n_cells;
    int64_t off_segs, off_xs, off_ys, off_zs, off_perm, off_keys_in, off_keys_out, off_vals_in,
        off_sort_tmp, sort_tmp_bytes, total_bytes;
    // Cartesian-grid check of a single-segment 2-D / 3-D plan (GridCheck):
    // the first index whose (y, z) differs from cell 0's (= nx), the first
    // whose z differs (= nx ny), a mismatch flag, and the plan's tag.  The
    // axes X (nx), Y (ny), Z (nz) are written over the keys_in scratch.
    GridCheck grid;
    int64_t reserved[10];
};
static_assert(sizeof(PlanHeader) <= 256, "plan header must fit in 256 bytes");

struct SegInfo {
    int64_t begin;        // first cell (global index)
    int64_t count;
    float lo[3];          // bounding box (float bits ordered as ints during the reduction)
    float hi[3];
    float inv_brick[3];   // quantisation levels per unit length (same on every axis)
    int32_t nb[3];        // quantisation levels per axis (<= 2^kMortonBits)
    int32_t pad;
};

struct PlanLayout {
    int64_t off_segs, off_xs, off_ys, off_zs, off_perm, off_keys_in, off_keys_out, off_vals_in,
        off_sort_tmp, sort_tmp_bytes, total;
};

size_t radix_sort_temp_bytes(int64_t n_cells);  // defined in plan.cu

inline PlanLayout plan_layout(int64_t n_cells, int32_t n_segments) {
    PlanLayout L;
    L.off_segs = 256;
    L.off_xs = L.off_segs + align256(int64_t(n_segments) * int64_t(sizeof(SegInfo)));
    L.off_ys = L.off_xs + align256(n_cells * 4);
    L.off_zs = L.off_ys + align256(n_cells * 4);
    L.off_perm = L.off_zs + align256(n_cells * 4);
    L.off_keys_in = L.off_perm + align256(n_cells * 4);
    L.off_keys_out = L.off_keys_in + align256(n_cells * 4);
    L.off_vals_in = L.off_keys_out + align256(n_cells * 4);
    L.off_sort_tmp = L.off_vals_in + align256(n_cells * 4);
    L.sort_tmp_bytes = int64_t(radix_sort_temp_bytes(n_cells));
    L.total = L.off_sort_tmp + align256(L.sort_tmp_bytes);
    return L;
}

// ---------------------------------------------------------------------------
// Map parameters as the kernels see them.
// ---------------------------------------------------------------------------
// Internal map bit, outside the public grf_map_bits: the field-mismatch loss
// of the calibration step and its gradient (grf_synth_mismatch), fused into
// the synthesis epilogue.
constexpr int32_t kMapMismatch = 1 << 16;

struct MapDev {
    int32_t bits;
    int32_t n_thr;
    float thr[GRF_MAX_THRESHOLDS];
    float values[GRF_MAX_THRESHOLDS + 1];
    float k_ref, phi0, phi1, phi_min, phi_max;
    float mu, sigma_inv;
    float* Y;
    float* K;
    uint8_t* F;
    float* P;
    // kMapMismatch: K = exp(Y), gY = g_scale (K - T) K, and per-unit sums of
    // (K - T)^2 in lpart (one entry per warp tile, or per block of the
    // split finalize), reduced afterwards into *loss / n_mean
    const float* T;
    float* G;
    double* lpart;
    double* loss;
    double inv_n_mean;
    float g_scale;        // 2 / n_mean (FP32, as the standalone loss kernel forms it)
    int32_t pad_;
};

// One realisation as the forward kernel sees it.
struct FwdDesc {
    const float4* hot;
    const float4* cold;
    const int32_t* kpref;
    int32_t n_pad;
    int32_t dim;
    float inv_tau1;       // 1 / (span limit of the light class, turns)
    float inv_tau2;       // 1 / (span limit of the medium class, turns)
    const float* xs;      // sorted coordinates of this realisation's segment
    const float* ys;
    const float* zs;
    const int32_t* perm;  // original (plan-global) index of each sorted cell
    int64_t perm_base;    // first plan-global index of the segment
    int64_t n_cells;
    MapDev map;
};

// Cartesian grid of a plan: cell n = i + nx (k + ny l) at (X_i, Y_k, Z_l).
struct GridGeom {
    int32_t nx, ny, nz;
    const float* X;
    const float* Y;
    const float* Z;
};

// Tables of one grid synthesis (workspace) as the prep kernel fills them.
struct GridPrep {
    const TableHeader* thdr;
    const float4* hot;
    const float4* cold;
    const float* X;
    const float* Y;
    const float* Z;
    int32_t nx, ny, nz, n_pad, nc, n_mt, n_kt, dim;
    int32_t form;          // 1: 3-D (B formed from ytab, wztab), 0: B tabulated in btab
    unsigned char* atab;   // x phasors: FP16 hi/lo tiles [n_mt][nc][2][128 x 64]
    unsigned char* btab;   // 2-D: B tiles [n_kt][nc][2][128 x 64]
    float2* ytab;          // 3-D: [nc][ny][32] y phasors
    float2* wztab;         // 3-D: [nc][nz][32] (amplitude, psi, z) phasors
};

// One grid synthesis as the tensor-core kernel sees it.
struct GridDesc {
    const unsigned char* atab;
    const unsigned char* btab;
    const float2* ytab;
    const float2* wztab;
    const TableHeader* thdr;
    int32_t nx, ny, nz, n_pad;
    int32_t nc;       // chunks of 32 modes
    int32_t fc;       // chunks per fold interval (1, 2 or 4)
    int32_t n_mt, n_kt, n_lt;
    int32_t pk_log2;  // (y, z) patch: 2^pk_log2 along y, 128 / 2^pk_log2 along z
    int64_t n_tiles;
    int32_t form;     // 1: B formed in shared memory from the staged table rows
    int32_t sa;       // stages of the copy ring
    int32_t a_stage;  // bytes per copy stage
    int32_t off_b;    // formed B ring (form)
    int32_t off_bar;  // barriers
    int32_t n_split;  // mode splits per tile (whole fold intervals each); > 1: partial fields in part
    int64_t n_items;  // tiles x splits
    float* part;      // [n_split][nx ny nz] partial fields (n_split > 1), summed by the finalize kernel
    MapDev map;
};

// Work tile of the batched launch: realisation r, tile index t inside it.
struct WorkItem {
    int32_t r;
    int32_t t;
};

// Batched workspace layout.
struct BatchHeader {
    uint32_t magic;
    int32_t n_items;
    int32_t n_work;
    int32_t tile_cells;
    int32_t cfg;          // kernel configuration index
    int32_t dim_max;
    int64_t off_desc, off_work, off_counter, total_bytes;
    int64_t reserved[24];
};
constexpr uint32_t kBatchMagic = 0x48435442u;  // "BTCH"

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files), all asynchronous on `stream`.
// Return cudaError_t as int.
// ---------------------------------------------------------------------------
int launch_synth_fwd(const FwdDesc& d, void* workspace, size_t ws_bytes, int32_t* status, void* stream);
// Entries of MapDev::lpart a launch of n cells may write (kMapMismatch).
int64_t mismatch_partials(int64_t n_cells);
// loss = (sum of the nb partials, fixed order) * inv_n, one block.
int launch_loss_sum(const double* part, int64_t nb, double inv_n, double* out, void* stream);

// Checked builds (-DGRF_CHECKED=1): device accesses skipped since the last
// call because an index read from device memory was out of range, per
// translation unit, then reset; ~0 if the counter cannot be read; always 0
// in release builds.
unsigned long long take_index_faults_fwd();
unsigned long long take_index_faults_bwd();
unsigned long long take_index_faults_plan();
// Warp tiles of single-field synthesis launches that took the general and the
// lattice path since the last call, then reset (synchronous); cudaError_t.
int take_path_counts(unsigned long long* general, unsigned long long* lattice);
// The same for the 3-D adjoint's warp tiles (synth_bwd.cu).
int take_bwd_path_counts(unsigned long long* general, unsigned long long* lattice);
size_t synth_workspace_bytes(int64_t n_cells);
int launch_synth_batched(const void* workspace, const BatchHeader& h, int32_t* status,
                         int32_t* counter, void* stream);
int fwd_tile_cells(int cfg);
int launch_map(const MapDev& m, int64_t n, const float* Y, void* stream);
int launch_bimap(const grf_bimap& m, int64_t n, const float* Y1, const float* Y2, uint8_t* F, float* P,
                 void* stream);
// tag: host-assigned plan number, stored with the grid check (GridCheck::tag)
int launch_plan(int32_t dim, int32_t n_segments, const int64_t* seg_offsets_host, const float* x,
                const float* y, const float* z, void* plan, const PlanLayout& L, uint64_t tag, void* stream);
// periodic_mask: bit c set when axis c is periodic (its frequency is rounded,
// so its dL/da reaches neither kappa, l nor R).
int launch_synth_bwd(const void* table, int64_t n_modes, int32_t dim, double sigma,
                     const double* ell, const double* rot, int32_t periodic_mask, const float* xs,
                     const float* ys, const float* zs,
                     const int32_t* perm, int64_t perm_base, int64_t n_cells, const float* gY,
                     const grf_grads& g, void* workspace, int32_t* status, void* stream);
size_t bwd_workspace_bytes(int64_t n_cells, int64_t n_modes, int32_t dim);
// Per-mode terms of the scalar gradients the adjoint's reduction writes
// (contrib rows: (A / sigma) dA, three l terms, nine R terms).
constexpr int kBwdContrib = 13;
// The adjoint's reduction and chain rule from per-mode partial sums:
// part[s][slot][5] = (sum g cos, sum g sin, sum g x sin, sum g y sin,
// sum g z sin) for s < splits (summed in increasing s), gpart[0 .. n_gpart)
// partial sums of g, contrib: kBwdContrib x n_pad doubles of scratch.
int launch_bwd_reduce(const void* table, int64_t n_modes, int32_t dim, double sigma, const double* ell,
                      const double* rot, int32_t periodic_mask, const grf_grads& g, double* part, int32_t splits,
                      double* gpart, int32_t n_gpart, double* contrib, void* stream);
// Tensor-core adjoint on a Cartesian grid in x-fastest order (synth_grid_bwd.cu):
// workspace bytes, the launch (scan, prep, tensor-core kernel, reduction) and
// the units computed since the last call (synchronous).
size_t bwd_grid_ws_bytes(int32_t nx, int32_t ny, int32_t nz, int64_t n_pad);
int launch_synth_bwd_grid(const void* table, int64_t n_modes, int32_t dim, const GridGeom& gg, const float* gY,
                          double sigma, const double* ell, const double* rot, int32_t periodic_mask,
                          const grf_grads& g, void* ws, int32_t* status, void* stream);
int take_grid_adj_units(unsigned long long* units);
int launch_mismatch(int64_t n, const float* K, const float* T, float* gY, double* loss, void* ws,
                    void* stream);
size_t mismatch_workspace_bytes(int64_t n);
int launch_mufu_probe(int32_t blocks, int32_t iters, float* sink, void* stream);
// Grid path (synth_grid.cu): workspace bytes of the tables, the launch (prep
// + tensor-core kernel), tiles computed since the last call (synchronous),
// and the MMA self-test.
size_t grid_ws_bytes(int32_t nx, int32_t ny, int32_t nz, int64_t n_pad);
// Loss partials (kMapMismatch) the grid path writes: one per epilogue warp per tile.
int64_t grid_loss_partials(int32_t nx, int32_t ny, int32_t nz);
// Tiles of 128 x 128 cells of a grid.
int64_t grid_tiles(int32_t nx, int32_t ny, int32_t nz);
int launch_synth_grid(const void* table, int64_t n_modes, int32_t dim, const GridGeom& gg, const MapDev& map,
                      void* ws, int32_t fc, int32_t* status, void* stream);
int take_grid_tiles(unsigned long long* tiles);
int launch_mma_probe(const uint16_t* A, const uint16_t* B, int32_t k_chunks, float* D, int32_t* status,
                     void* stream);
int launch_grid_check(int32_t dim, int64_t n, const float* x, const float* y, const float* z, void* plan,
                      const PlanLayout& L, void* stream);
int launch_selftest_wait(uint64_t limit_ns, int32_t* status, void* stream);
void count_launches(int64_t n);
// Record `message` as the calling thread's last error and return `code`.
int set_error(int code, const char* message);
// Allocation point of the host code: throws std::bad_alloc while injected
// failures remain (grf_debug_inject_alloc_failures); ABI entry points turn
// it into GRF_ENOMEM.
void alloc_point();

}  // namespace grf
