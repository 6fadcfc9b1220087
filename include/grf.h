/*
 * grf.h -- C ABI of the GB300 spectral Gaussian-random-field library.
 *
 * Method (Icardi et al., "Computational framework for complex flow and
 * transport in heterogeneous porous media", arXiv 2212.10961):
 *   Sec. 4.1, Eq. (DiscreteFT): a Gaussian random field evaluated directly at
 *     arbitrary cell centres as a finite sum of N cosine modes (no FFT), with
 *     frequencies drawn from the spectral density of the covariance and a
 *     per-axis rescaling of frequency space for anisotropy;
 *   Appendix A, Eqs. (gauSpe), (expSpe), (matSpe): Gaussian, exponential and
 *     Matern covariances and their spectra;
 *   Sec. 3.1 and Sec. 4.1 / Appendix B: scaling to mean and variance
 *     (lognormal permeability), single truncation rule (facies thresholds),
 *     facies values; Appendix B lists the user parameters mirrored by
 *     grf_params.
 *
 * Real form used everywhere (see grf_gen_modes for the reading of the
 * paper's complex "+ i sum sin"):
 *     Y(x) = mu + sum_{j<N} A_j cos(2 pi (a_j . x + psi_j)),
 *     A_j = sigma rho_j,  a_j = kappa_j / (2 pi l)  (per axis).
 *
 * Conventions for every entry point:
 *   - Return value: GRF_OK (0) or a negative GRF_E* code.  No C++ exception
 *     crosses the ABI.  grf_last_error() gives a message for the calling
 *     thread's last failure.
 *   - Ownership: the caller allocates and frees every buffer.  The library
 *     allocates no device memory; it may allocate small host buffers.
 *   - "device" pointers are CUDA global-memory addresses of the current
 *     device; "host" pointers are ordinary process memory.  A `stream`
 *     argument is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued asynchronously on that stream; host
 *     buffers handed to an asynchronous copy must stay valid until the stream
 *     reaches it.
 *   - Cell centres are structure-of-arrays float32: x[i], y[i], z[i];
 *     y is ignored (may be NULL) when dim < 2 and z when dim < 3.
 */
#ifndef GRF_H
#define GRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* Status codes                                                         */
/* ------------------------------------------------------------------ */
#define GRF_OK 0
#define GRF_EINVAL (-1)     /* invalid argument: NULL pointer, size, range or order */
#define GRF_EWORKSPACE (-2) /* a caller buffer is smaller than required */
#define GRF_ECUDA (-3)      /* a CUDA runtime call or kernel launch failed */
#define GRF_ETIMEOUT (-4)   /* a bounded device-side wait expired; kernel returned early */
#define GRF_ENOMEM (-5)     /* a host allocation failed */
#define GRF_EDEVICE (-6)    /* a device-side check failed (see grf_read_status) */

/* Message describing the calling thread's most recent failure ("" if none).
 * The pointer stays valid until the next library call on the same thread. */
const char *grf_last_error(void);

/* Library version string, e.g. "grf-gb300 1.0". */
const char *grf_version(void);

/* ------------------------------------------------------------------ */
/* Parameters (Appendix B: correlation, Kmean, Ksigma, Lcorr, nu, nfreq, */
/* disableY/disableZ)                                                   */
/* ------------------------------------------------------------------ */
enum grf_family {
    GRF_GAUSSIAN = 0,    /* Appendix A, Eq. (gauSpe) */
    GRF_EXPONENTIAL = 1, /* Appendix A, Eq. (expSpe); equals Matern nu = 1/2 */
    GRF_MATERN = 2       /* Appendix A, Eq. (matSpe) */
};

typedef struct grf_params {
    int32_t family;   /* enum grf_family */
    int32_t dim;      /* 1, 2 or 3 (Appendix B disableY / disableZ) */
    double nu;        /* Matern smoothness, > 0 (read only for GRF_MATERN) */
    double sigma2;    /* variance of Y ("Ksigma"), > 0 */
    double mean;      /* mean of Y ("Kmean") */
    double ell[3];    /* correlation length per axis ("Lcorr"), > 0; ell[c], c < dim */
    int64_t n_modes;  /* N ("nfreq"), 1 .. GRF_MAX_MODES */
    uint64_t seed;    /* generator key */
    uint32_t stream;  /* independent generator stream (e.g. 2nd field of a pair) */
    uint32_t reserved;/* must be 0 */
    double period[3]; /* Appendix B `periodic`: L_c > 0 makes the field repeat with
                         period L_c along axis c (frequencies moved to the nearest
                         multiple of 1/L_c); 0 = not periodic */
    double rot[9];    /* transform of the anisotropy axes (Sec. 4.1: the per-axis
                         rescaling of frequency space, extended to rotations and
                         general transformation matrices): row-major R, C(r) = sigma^2
                         rho(|diag(1/l) R r|).  A rotation (rows = principal axes) or
                         any invertible matrix; the leading dim x dim block is used.
                         All zeros = no transform. */
} grf_params;

#define GRF_MAX_MODES (1 << 24)

/* ------------------------------------------------------------------ */
/* S1: drawing the modes (host, FP64)                                   */
/* ------------------------------------------------------------------ */
/*
 * Host FP64 mode set, arrays allocated by the caller with n entries
 * (n * dim for kappa and a, row-major: element (j, c) at j * dim + c).
 */
typedef struct grf_modes {
    int64_t n;      /* number of modes, must equal params->n_modes */
    int32_t dim;    /* must equal params->dim */
    int32_t reserved;
    double *kappa;  /* standardised wave-vectors (k_c * l_c) */
    double *rho;    /* amplitude weights sqrt((W^2 + W'^2) / N) */
    double *psi;    /* phases in turns, in (-1/2, 1/2] */
    double *a;      /* frequencies in turns per unit length, kappa_c / (2 pi l_c) */
    double *amp;    /* amplitudes A_j = sigma * rho_j */
} grf_modes;

/*
 * grf_gen_modes -- draw the N modes of one realisation.
 * Sec. 4.1 (Eq. DiscreteFT, rescaling of frequency space) and Appendix A.
 *
 * Readings: the field is the real sum W_j cos + W'_j sin with exactly N
 * terms; a_j are i.i.d. draws from the spectral density normalised to a
 * probability density, so the amplitude is sigma/sqrt(N) times the Gaussian
 * weights (exact covariance for every N).  Standardised wave-vectors:
 * Gaussian kappa_c = sqrt(pi/2) z_c; Matern(nu) (exponential: nu = 1/2)
 * kappa = z sqrt(2 nu / w), w ~ chi^2 with 2 nu degrees of freedom.
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with
 * key = (seed lo, seed hi) and counter = (j lo, block, stream, j hi);
 * per mode, normals 0, 1 are W, W'; normals 2 .. 1+dim are z; for integer
 * 2 nu <= 32, w sums the squares of the next 2 nu normals; otherwise
 * w = 2 Gamma(nu) by Marsaglia-Tsang (attempt t: first normal of block
 * 64 + 2t, first uniform of block 65 + 2t; nu < 1 boosted with the first
 * uniform of block 63).  A block's two 64-bit words u give uniforms
 * (floor(u / 2^12) + 1/2) 2^-52; Box-Muller turns them into two normals.
 *
 * Rotation (p->rot non-zero): a_j = R^T u_j with u_jc = kappa_jc / (2 pi l_c).
 * Periodic axes (p->period[c] > 0, applied after the rotation):
 * a_jc = floor(a_jc L_c + 1/2) / L_c, so that Y(x + L_c e_c) = Y(x); kappa
 * keeps the drawn value.
 *
 * Arguments: p (host, read), out (host, arrays written).  Returns GRF_EINVAL
 * for bad parameters or mismatched out->n / out->dim, GRF_OK otherwise.
 * Deterministic: the same (seed, stream, j) always gives the same mode j,
 * whatever N.
 */
int grf_gen_modes(const grf_params *p, grf_modes *out);

/*
 * grf_reparam_modes -- amplitudes and frequencies of given standardised modes.
 * Sec. 4.1: the field is scaled to its variance (A_j = sigma rho_j) and the
 * frequency space is rescaled per axis for anisotropy (u_jc = kappa_jc /
 * (2 pi l_c)), extended to an axis transform R (a_j = R^T u_j, p->rot) and
 * to the Appendix B `periodic` option (a_jc = floor(a_jc L_c + 1/2) / L_c on
 * every axis with p->period[c] = L_c > 0, after the transform).  This is the
 * second half of grf_gen_modes, for callers that hold kappa_j and rho_j as
 * parameters of their own (calibration, inversion) instead of drawing them.
 *
 * Arguments: p (host, read: sigma2, ell, rot, period, n_modes, dim); m
 * (host): m->kappa [n*dim] and m->rho [n] are read, m->amp [n] and m->a
 * [n*dim] written, m->psi is not touched.  Returns GRF_EINVAL for bad
 * parameters, mismatched m->n / m->dim, a NULL array or a non-finite kappa
 * or rho; GRF_OK otherwise.  Same arithmetic as grf_gen_modes, so modes drawn
 * there reparameterise to bit-identical amp and a.
 */
int grf_reparam_modes(const grf_params *p, grf_modes *m);

/* ------------------------------------------------------------------ */
/* Device mode table                                                    */
/* ------------------------------------------------------------------ */
/*
 * The device table is an opaque, 256-byte aligned image built on the host by
 * grf_pack_table and copied to the device by grf_upload_table.  It holds,
 * per mode, FP32 angular frequencies 2 pi a, the amplitude A, the frequency
 * and phase as FP32 hi/lo pairs (for the compensated phase split), the
 * original mode index, and a per-extent table of how many modes need the
 * compensated path.  Modes are stored in decreasing order of |a|_1; the sum
 * is order independent.  Every mode at an odd position is stored in the
 * equivalent form (-A, psi + 1/2), so that a mean offset of the hardware
 * cosine's error cancels over the sum instead of growing with sqrt(N).
 */
size_t grf_table_bytes(int64_t n_modes);

/* Build the table image of modes m (A = m->amp, a = m->a, psi = m->psi)
 * into host memory `host_table` of `bytes` >= grf_table_bytes(m->n).
 * m->kappa may be NULL; when given it is stored too, for the adjoint's
 * chain rule to l, R and kappa (grf_synth_backward).  m->rho is not read.
 * GRF_EWORKSPACE if too small, GRF_EINVAL for NULL arrays or bad sizes. */
int grf_pack_table(const grf_modes *m, void *host_table, size_t bytes);

/* Enqueue the host->device copy of a packed table (cudaMemcpyAsync).
 * host_table must stay valid until the copy has run (pinned memory makes
 * the copy truly asynchronous).  dev_table must be 256-byte aligned. */
int grf_upload_table(const void *host_table, void *dev_table, size_t bytes, void *stream);

/* ------------------------------------------------------------------ */
/* Mode prefetcher (many realisations of one parameter set)             */
/* ------------------------------------------------------------------ */
/*
 * Monte-Carlo runs draw a new realisation of the same field many times
 * (Sec. 4.1: a realisation is fixed by its parameters and seed).  The
 * prefetcher draws (grf_gen_modes) and packs (grf_pack_table, with kappa)
 * realisation k = 0, 1, 2, ... with seed p->seed + k on `threads` host
 * worker threads of its own, up to `depth` realisations ahead of use, into a
 * ring of `depth` caller-provided staging buffers (host_slots[s], slot_bytes
 * >= grf_table_bytes(p->n_modes) each; pinned memory makes the uploads
 * asynchronous).  The caller's thread then only enqueues uploads.
 *
 * grf_prefetch_create: p is copied; the current device is recorded and made
 * current on the workers.  GRF_EINVAL for bad parameters, depth outside
 * [2, 64], threads outside [1, 64] or a NULL slot; GRF_EWORKSPACE for slots
 * too small; GRF_ECUDA if events cannot be created.
 * grf_prefetch_next: waits (on the host) for the next realisation in order,
 * enqueues its upload into dev_table (device, 256-byte aligned, bytes >=
 * grf_table_bytes) on `stream` and returns its seed in *seed_out (may be
 * NULL).  A slot is reused only after its upload has run (an event recorded
 * on `stream`).  A worker's failure (e.g. a sampler that does not accept) is
 * returned by the next call with its message.  Calls on one prefetcher must
 * come from one thread at a time.
 * grf_prefetch_destroy: stops and joins the workers, waits for uploads still
 * pending from the staging buffers (the caller may free them afterwards) and
 * frees the prefetcher.  NULL is ignored.
 */
typedef struct grf_prefetch grf_prefetch;
int grf_prefetch_create(const grf_params *p, int32_t depth, int32_t threads, void *const *host_slots,
                        size_t slot_bytes, grf_prefetch **out);
int grf_prefetch_next(grf_prefetch *pf, void *dev_table, size_t bytes, void *stream, uint64_t *seed_out);
int grf_prefetch_destroy(grf_prefetch *pf);

/* ------------------------------------------------------------------ */
/* Cell plan (spatial binning of arbitrary cell centres)                */
/* ------------------------------------------------------------------ */
/*
 * The paper evaluates Eq. (DiscreteFT) at the cell centres of an arbitrary
 * mesh (Sec. 4.1: Cartesian grids are treated as unstructured).  The plan
 * is a permutation that groups nearby cells so that each warp works on a
 * compact set, which keeps the FP32 phase split accurate.  It is built on
 * the device once per mesh (bounding box, Morton brick keys, stable radix
 * sort, gather of sorted SoA coordinates) and reused for every realisation
 * on that mesh.
 *
 * Several independent meshes ("segments", e.g. the grids of an ensemble)
 * can share one plan: seg_offsets (host, n_segments + 1 entries, ascending,
 * seg_offsets[0] = 0) delimit their cells in x/y/z.
 */
size_t grf_plan_bytes(int64_t n_cells, int32_t n_segments);

/* x, y, z: device float32 arrays of seg_offsets[n_segments] cells.
 * plan: device buffer, 256-byte aligned, plan_bytes >= grf_plan_bytes().
 * The input arrays are read only while the stream runs the planning
 * kernels; the plan keeps its own sorted copy of the coordinates.
 * Coordinates must be finite (GRF_EDEVICE via grf_read_status otherwise). */
int grf_plan_cells(int32_t dim, int32_t n_segments, const int64_t *seg_offsets,
                   const float *x, const float *y, const float *z, void *plan,
                   size_t plan_bytes, void *stream);

/*
 * grf_release -- drop the library's host-side record of a plan (built by
 * grf_plan_cells) or of a batch workspace (prepared by grf_batch_prepare).
 * The library keeps one small record per such buffer for the life of the
 * process; release it before the caller frees or reuses the buffer, so that
 * a stale pointer passed later is rejected (GRF_EINVAL) instead of being
 * read as a plan.  The device buffer itself is untouched.  Pointers the
 * library does not know are ignored.  Returns GRF_OK.
 */
int grf_release(const void *buffer);

/* Device status word of a plan (0 = no device-side error).  Synchronises
 * the stream.  Bits: 1 = non-finite coordinate, 2 = bounded wait expired,
 * 4 = table/plan mismatch detected on the device. */
int grf_read_status(const void *plan, int32_t *status_out, void *stream);

/* ------------------------------------------------------------------ */
/* S2-S4: field synthesis with fused property maps                      */
/* ------------------------------------------------------------------ */
#define GRF_MAX_THRESHOLDS 15

enum grf_map_bits {
    GRF_MAP_Y = 1,         /* write the Gaussian field Y */
    GRF_MAP_LOGNORMAL = 2, /* K = k_ref exp(Y)  (Sec. 4.1, log-permeability field) */
    GRF_MAP_FACIES = 4,    /* label = #{m : Y > t_m}  (Sec. 3.1 single truncation rule) */
    GRF_MAP_VALUES = 8,    /* prop = values[label]  (Appendix B `values`) */
    GRF_MAP_POROSITY = 16  /* prop = clamp(phi0 + phi1 (Y - mu)/sigma, phi_min, phi_max) */
};

typedef struct grf_map {
    int32_t bits;          /* OR of grf_map_bits; VALUES and POROSITY exclusive */
    int32_t n_thresholds;  /* 0 .. GRF_MAX_THRESHOLDS (FACIES / VALUES) */
    float thresholds[GRF_MAX_THRESHOLDS]; /* ascending, in Y units */
    float values[GRF_MAX_THRESHOLDS + 1]; /* value per facies (VALUES) */
    float k_ref;           /* LOGNORMAL prefactor (1 = plain exp) */
    float phi0, phi1, phi_min, phi_max;   /* POROSITY */
} grf_map;

/* Device outputs in the caller's original cell order; an output may be
 * NULL when its bit is not requested, and every output may be NULL when
 * there are no cells to write (an empty plan or segment, n = 0). */
typedef struct grf_outputs {
    float *Y;         /* GRF_MAP_Y */
    float *K;         /* GRF_MAP_LOGNORMAL */
    uint8_t *facies;  /* GRF_MAP_FACIES */
    float *prop;      /* GRF_MAP_VALUES or GRF_MAP_POROSITY */
} grf_outputs;

/*
 * grf_synth_field -- Y_i = mu + sum_j A_j cos(2 pi (a_j . x_i + psi_j)) at
 * every cell of segment `segment` of `plan`, followed by the requested maps,
 * all in one kernel.  Sec. 4.1, Eq. (DiscreteFT); maps Sec. 3.1, Sec. 4.1,
 * Appendix B.
 *
 * table: device table (grf_upload_table) of p->n_modes modes, dim p->dim.
 * p: host; mean and sigma2 are read (porosity standardisation), the rest is
 * checked against the table.  map, out: host structs of device pointers.
 * workspace: optional device scratch (NULL or ws_bytes too small: no mode
 * split); see grf_synth_workspace_bytes.  Calls that share a workspace must
 * be ordered on one stream.
 * Arithmetic: FP32 with a compensated phase split (per-warp origin with
 * hi/lo frequencies, exact path for modes whose phase span is large) and
 * compensated accumulation; the hardware cosine.  Results agree with the
 * FP64 definition to a few 1e-6 sigma (max-abs).
 */
int grf_synth_field(const void *table, const grf_params *p, const void *plan, int32_t segment,
                    const grf_map *map, const grf_outputs *out, void *workspace, size_t ws_bytes,
                    void *stream);

/* Workspace that lets grf_synth_field split the modes of a segment of
 * n_cells cells over up to 8 groups of blocks (8 float2 per cell).  The split
 * is used only when the segment has too few cell tiles to fill the GPU; the
 * per-group partial sums are combined in a fixed order, so results do not
 * depend on it beyond FP32 rounding and are reproducible. */
size_t grf_synth_workspace_bytes(int64_t n_cells);

/*
 * Cartesian grids (tensor-core path).  When a single-segment 2-D or 3-D plan
 * holds the cells of a Cartesian grid handed over x-fastest -- cell
 * n = i + nx (k + ny l) at (X_i, Y_k, Z_l) for axes X, Y, Z of any spacing,
 * with ny >= 2 -- grf_plan_cells records the grid (a check that runs with the
 * planning kernels).  grf_synth_field on such a plan (with the grid path
 * on, see grf_debug_grid_path), with a field of the plan's
 * dimension and a workspace of at least
 * grf_synth_grid_workspace_bytes() bytes, then evaluates Eq. (DiscreteFT) as
 * a matrix product on the tensor cores: every term factorises into an x
 * phasor and a (y, z) phasor, so a block of 128 x-cells by 128 (y, z)-cells
 * is a real product over K = 2N (Sec. 4.1 term by term, no approximation).
 * Operands are split into FP16 hi + lo pairs (three products per term) and
 * the FP32 partial sums of a few chunks of modes are folded into running
 * sums: results agree with the FP64 definition to a few 1e-6 sigma, as on the
 * general path.  Outputs
 * and maps are those of the general path, in the caller's cell order.
 *
 * grf_synth_mismatch takes the same path on such a plan when the part of its
 * workspace after the loss partials (grf_synth_mismatch_workspace_bytes(n) -
 * grf_synth_workspace_bytes(n) bytes) holds grf_synth_grid_workspace_bytes().
 *
 * grf_synth_grid_workspace_bytes -- workspace bytes the grid path needs for
 * `plan` (segment 0) and a table of n_modes modes, or 0 when the plan is not
 * such a grid (or is unknown), or when those tables would exceed
 * max(1 GB, 64 bytes per cell) (N far above the cell count: such calls take
 * the CUDA-core kernels).  The first query (or synthesis) of a new plan
 * waits on the host for that plan's own kernels to finish.
 * grf_plan_grid_shape -- the plan's grid (nx, ny, nz), or zeros.  Same wait.
 * GRF_EINVAL for NULL pointers or an unknown plan.
 */
size_t grf_synth_grid_workspace_bytes(const void *plan, int32_t segment, int64_t n_modes);
int grf_plan_grid_shape(const void *plan, int32_t *nx, int32_t *ny, int32_t *nz);

/*
 * grf_map_property -- the maps of grf_synth_field applied to an existing
 * field Y (device, n values), writing `out` in the same order.  Memory bound.
 * mean, sigma: the Gaussian field's mean and standard deviation (porosity).
 */
int grf_map_property(const grf_map *map, double mean, double sigma, int64_t n, const float *Y,
                     const grf_outputs *out, void *stream);

/*
 * Bitruncated (pluri-Gaussian) facies, Sec. 3.1 and Appendix B `bitruncated`
 * / `thresholds2`: two independent Gaussian fields Y1, Y2 (e.g. the same
 * parameters drawn on generator streams 0 and 1) are binned by ascending
 * thresholds t (on Y1) and s (on Y2); region (i, j) with
 * i = #{m : Y1 > t_m}, j = #{m : Y2 > s_m} is merged into facies rule[i][j].
 */
typedef struct grf_bimap {
    int32_t n_t;                                            /* 0 .. GRF_MAX_THRESHOLDS */
    int32_t n_s;                                            /* 0 .. GRF_MAX_THRESHOLDS */
    float t[GRF_MAX_THRESHOLDS];                            /* ascending, Y1 units */
    float s[GRF_MAX_THRESHOLDS];                            /* ascending, Y2 units */
    uint8_t rule[GRF_MAX_THRESHOLDS + 1][GRF_MAX_THRESHOLDS + 1]; /* facies of region (i, j) */
    float values[256];                                      /* prop = values[facies] */
} grf_bimap;

/* Facies (device uint8, required) and optionally prop (device float32,
 * NULL to skip) of n cells from the two fields Y1, Y2 (device float32, same
 * cell order).  Memory bound. */
int grf_map_bitruncated(const grf_bimap *map, int64_t n, const float *Y1, const float *Y2,
                        uint8_t *facies, float *prop, void *stream);

/* ------------------------------------------------------------------ */
/* S5: adjoint                                                          */
/* ------------------------------------------------------------------ */
/* Device FP64 gradient outputs (original mode order j of grf_gen_modes).
 * With u_j = kappa_j / (2 pi l) the frequencies before the axis transform and
 * e_j = M dL/da_j, where M zeroes the components of periodic axes (their
 * rounded frequency is locally constant in kappa, l and R, so dL/da of a
 * periodic axis reaches none of them; without periodic axes e_j = dL/da_j): */
typedef struct grf_grads {
    double *dA;     /* [N]      dL/dA_j   = sum_i g_i cos theta_ij */
    double *dpsi;   /* [N]      dL/dpsi_j = -2 pi A_j sum_i g_i sin theta_ij */
    double *da;     /* [N*dim]  dL/da_jc  = -2 pi A_j sum_i g_i sin theta_ij x_ic */
    double *dmu;    /* [1]      sum_i g_i */
    double *dsigma; /* [1]      sum_j (A_j / sigma) dL/dA_j = sum_j rho_j dL/dA_j */
    double *dell;   /* [dim]    -sum_j (u_jc / l_c) (R e_j)_c (R = I without a transform) */
    double *drot;   /* [dim*dim] or NULL: dL/dR_cd = sum_j u_jc e_jd, R as a free
                       row-major matrix (only meaningful with a transform) */
    double *dsigma2;/* [1] or NULL: dL/d(sigma^2) = dsigma / (2 sigma) */
    double *drho;   /* [N] or NULL:     dL/drho_j = sigma dL/dA_j */
    double *dkappa; /* [N*dim] or NULL: dL/dkappa_jc = (R e_j)_c / (2 pi l_c) */
    const double *gscale; /* [1] device, or NULL for 1: every output above is
                       multiplied by *gscale (the gradient of gscale * L; an
                       upstream factor read on the device, e.g. by autograd) */
} grf_grads;

/* Workspace for grf_synth_backward on n_cells cells and n_modes modes. */
size_t grf_backward_workspace_bytes(int64_t n_cells, int64_t n_modes, int32_t dim);

/*
 * grf_backward_grid_workspace_bytes -- workspace bytes grf_synth_backward
 * needs to take the tensor-core grid adjoint on `plan` (segment 0, a
 * Cartesian grid in x-fastest order, dim >= 2) with n_modes modes: the
 * per-mode partials, the tables of x, y and z phasors and the FP16 tiles of
 * gY.  0 when the plan is not such a grid, its check is unresolved only
 * through a failed event, the arguments are invalid, or the tables would
 * exceed max(1 GB, 64 bytes per cell) (the CUDA-core adjoint serves it).
 */
size_t grf_backward_grid_workspace_bytes(const void *plan, int32_t segment, int64_t n_modes);

/*
 * grf_synth_backward -- gradients of a loss L with respect to the mode
 * amplitudes, phases and frequencies, the mean, sigma and the correlation
 * lengths, given gY = dL/dY (device float32, original cell order, cells of
 * segment `segment` of `plan`).  Derivative of Eq. (DiscreteFT) with the
 * reparameterisation of Sec. 4.1 (grf_reparam_modes): A = sigma rho,
 * a = R^T kappa / (2 pi l), periodic axes rounded.  p gives sigma, l, R and
 * the periodic axes of the chain rule.  u_j is read from the kappa the table
 * was packed with; a table packed without kappa uses u_j = R^-T a_j instead,
 * which is the same unless an axis is periodic.
 * The sines and cosines are recomputed, never stored.  Per-block FP64
 * partials go to `workspace` and are reduced in a fixed order, so results
 * are deterministic.  All non-optional outputs in `g` are written (device).
 * Grid path: when the plan is a Cartesian grid in x-fastest order (dim >= 2,
 * one segment), the grid path is enabled for it (grf_debug_grid_path) and
 * ws_bytes >= grf_backward_grid_workspace_bytes(), the per-mode sums are
 * matrix products on the tensor cores: D_j(k, l) = sum_i e^{2 pi i a_jx X_i}
 * g(i, k, l) over the x cells (FP16 hi + lo operands, three products per
 * term, FP32 accumulators over 64 x cells), contracted with the y and z
 * phasors per mode on the CUDA cores.  Otherwise ws_bytes must be at least
 * grf_backward_workspace_bytes() (GRF_EWORKSPACE).
 */
int grf_synth_backward(const void *table, const grf_params *p, const void *plan, int32_t segment,
                       const float *gY, const grf_grads *g, void *workspace, size_t ws_bytes,
                       void *stream);

/*
 * grf_synth_mismatch -- the forward half of a calibration step in one pass:
 * the field Y (Eq. DiscreteFT, as grf_synth_field) at every cell of segment
 * `segment` of `plan`, K = exp(Y), the field-mismatch loss
 *     L = sum_i (K_i - T_i)^2 / n_mean
 * against the target T = K_target, and its gradient gY_i = dL/dY_i =
 * 2 (K_i - T_i) K_i / n_mean, formed in the synthesis kernel's epilogue
 * (no K round trip through memory).  gY then feeds grf_synth_backward.
 * n_mean: the number of cells of the mean; 0 means the segment's own count.
 * A field sharded over processes passes the total over all shards, so that
 * the shards' losses and gradients add up to those of the whole field.
 *
 * K_target, gY: device float32 in the caller's original cell order; loss:
 * device double[1], reduced in a fixed order (deterministic).  Y_out, K_out:
 * optional device float32 outputs of the field and of K (NULL: not written).
 * workspace: device scratch of grf_synth_mismatch_workspace_bytes(n) bytes,
 * 256-byte aligned (the loss partial sums first; a smaller buffer that still
 * holds them disables the mode split).  Same arithmetic as grf_synth_field
 * followed by grf_mismatch_grad with n = n_mean: gY is identical, the loss
 * equal up to the order of the FP64 sum.  GRF_EINVAL for n_mean < the
 * segment's cell count or NULL buffers, GRF_EWORKSPACE for a workspace too
 * small for the loss partials.
 */
int grf_synth_mismatch(const void *table, const grf_params *p, const void *plan, int32_t segment,
                       const float *K_target, int64_t n_mean, float *gY, double *loss, float *Y_out,
                       float *K_out, void *workspace, size_t ws_bytes, void *stream);
size_t grf_synth_mismatch_workspace_bytes(int64_t n_cells);

/* Workspace for grf_mismatch_grad on n cells. */
size_t grf_mismatch_workspace_bytes(int64_t n);

/*
 * grf_mismatch_grad -- field-mismatch loss L = mean_i (K_i - T_i)^2 of a
 * lognormal field K = exp(Y) against a target T, and gY = dL/dY =
 * 2 (K - T) K / n (device float32).  loss: device double[1], reduced
 * deterministically through `workspace`.
 */
int grf_mismatch_grad(int64_t n, const float *K, const float *K_target, float *gY, double *loss,
                      void *workspace, size_t ws_bytes, void *stream);

/*
 * grf_mismatch_grad_noalloc -- the same loss and gradient as
 * grf_mismatch_grad, for callers that cannot allocate device memory at the
 * call site: a plug-in that must not touch its host application's
 * allocator, or a process whose device-memory budget is fixed once at
 * start-up.  No counterpart in the paper: it only changes where the
 * per-block partial sums live.
 *
 * The call itself makes CUDA runtime calls (it looks up the scratch array's
 * address) and enqueues two kernels on `stream`; like any CUDA call it must
 * not be made from inside a host callback (cudaLaunchHostFunc or a stream
 * callback), where CUDA calls are not allowed.
 *
 * The partial sums go to a fixed array inside the library,
 * GRF_NOALLOC_MAX_BLOCKS doubles (512 KiB) in device memory, which every GPU
 * that loads the library keeps until the process exits.  n may therefore be
 * at most GRF_NOALLOC_MAX_CELLS (134,217,728); larger n returns GRF_EINVAL
 * before any device work.  Every call looks up the array's device address in
 * the current device's context (cudaGetSymbolAddress), so a context reset
 * between calls is harmless; a device's first call also loads the library's
 * device code there: make that first call outside any CUDA-graph stream
 * capture.  All calls share the one array, so calls that can overlap on the
 * GPU (different streams, no ordering between them) race and may return
 * wrong losses: order them on one stream.  Nothing in the array needs to
 * start at zero; every call writes all the entries it reads.  Arguments and
 * results are those of grf_mismatch_grad.
 */
#define GRF_NOALLOC_MAX_BLOCKS 65536
#define GRF_NOALLOC_MAX_CELLS (134217728LL)
int grf_mismatch_grad_noalloc(int64_t n, const float *K, const float *K_target, float *gY,
                              double *loss, void *stream);

/* ------------------------------------------------------------------ */
/* S6: batched ensembles (many realisations, one persistent launch)     */
/* ------------------------------------------------------------------ */
typedef struct grf_batch_item {
    const void *table;  /* device table of this realisation */
    int64_t n_modes;
    int32_t dim;
    int32_t segment;    /* plan segment holding this realisation's cells */
    double mean;
    double sigma;
    grf_map map;
    grf_outputs out;    /* device outputs, segment-local original order */
} grf_batch_item;

/* Workspace for a batch of n_items realisations whose plan covers n_cells. */
size_t grf_batch_workspace_bytes(int32_t n_items, int64_t n_cells);

/*
 * grf_batch_prepare -- copy the descriptors of n_items realisations and a
 * cost-ordered work list into `workspace` (H2D from host_staging, which
 * must hold grf_batch_workspace_bytes() bytes and stay valid until the copy
 * has run).  tile_cells selects the cells per work item, one warp's tile
 * (0 = library choice, otherwise 128, 256 or 512: 4, 8 or 16 cells per
 * lane).  Call once per batch layout.
 */
int grf_batch_prepare(int32_t n_items, const grf_batch_item *items, const void *plan,
                      int32_t tile_cells, void *workspace, size_t ws_bytes, void *host_staging,
                      void *stream);

/*
 * grf_batch_autotune -- choose the work-tile shape for a batch by timing it.
 * Every candidate (256, 512 and 128 cells per warp tile: 8, 16 or 4 cells
 * per lane) is prepared and launched twice on `stream` (the second
 * launch timed with CUDA events), the fastest is written to *tile_cells and
 * its time in milliseconds to *best_ms, and `workspace` is left prepared for
 * it.  Results are cached in the process by batch signature (item count,
 * total cells, total cell-modes, plan dimension), so repeated calls for the
 * same layout only re-prepare.  Synchronises the stream; the outputs of the
 * items are overwritten.  Same buffers as grf_batch_prepare.
 */
int grf_batch_autotune(int32_t n_items, const grf_batch_item *items, const void *plan,
                       void *workspace, size_t ws_bytes, void *host_staging, void *stream,
                       int32_t *tile_cells, float *best_ms);

/*
 * grf_batch_launch -- one persistent launch synthesising every prepared
 * realisation (Eq. DiscreteFT and maps, as grf_synth_field).  Warps pull
 * work tiles from a counter in `workspace`, which this call resets first
 * (a memset node plus one kernel node: safe to capture in a CUDA graph
 * and replay).
 */
int grf_batch_launch(void *workspace, void *stream);

/*
 * grf_selftest_wait -- exercise the bounded-wait failure path on the device.
 * Launches one block that waits on a shared-memory mbarrier nothing ever
 * completes, with the same bounded wait the synthesis kernels use but a
 * limit of `limit_us` microseconds (1 .. 2,000,000).  The block records the
 * expiry in a device status word and returns; the call synchronises the
 * stream and returns GRF_ETIMEOUT when the wait expired as designed (GRF_OK
 * would mean the wait completed, which cannot happen).  The context stays
 * usable afterwards.  `status_dev` is a caller device int32 (set to 2).
 */
int grf_selftest_wait(int32_t limit_us, int32_t *status_dev, void *stream);

/*
 * Checked builds (the stand-in for a memory sanitizer).  The same sources
 * compiled with -DGRF_CHECKED=1 give libgrf_checked.so, with the same entry
 * points: before a kernel uses an index it read from device memory as an
 * address (an entry of a plan's permutation, a radix-sort scatter position),
 * it tests the index against the array it addresses; an index out of range
 * is counted and its access skipped instead of reading or writing out of
 * bounds.  Nothing else changes.
 *
 * grf_checked_build -- 1 for the checked library, 0 for the release one.
 *
 * grf_take_index_faults -- the number of accesses skipped since the last
 * call (and resets the count).  Synchronises the device; *count_out is
 * always 0 in the release library.  GRF_EINVAL for a NULL pointer,
 * GRF_ECUDA if the device counter cannot be read.
 */
int grf_checked_build(void);
int grf_take_index_faults(int64_t *count_out);

/* ------------------------------------------------------------------ */
/* Measurement helpers                                                  */
/* ------------------------------------------------------------------ */
/* Device properties used by the roofline: SM count and max SM clock (kHz). */
int grf_device_info(int32_t *sm_count, int32_t *sm_clock_khz);

/* Number of kernels the library launched on this process so far (all
 * entry points).  Used to report kernel counts in benchmarks. */
int64_t grf_launch_count(void);

/*
 * grf_take_path_counts -- warp tiles of 2-D and 3-D syntheses
 * (grf_synth_field, grf_synth_mismatch, grf_batch_launch) since the last
 * call that took the
 * general path and the lattice path (lanes holding 4-cell rows of one
 * Cartesian grid, see the synthesis kernel), then resets both.  A tile split
 * over mode groups counts once per group.  Synchronises the device.
 * GRF_EINVAL for NULL pointers, GRF_ECUDA if the counters cannot be read.
 */
int grf_take_path_counts(int64_t *general_warps, int64_t *lattice_warps);

/*
 * grf_take_adjoint_path_counts -- the same for the 3-D adjoint
 * (grf_synth_backward): (warp, cell tile) pairs since the last call that took
 * the general path and the lattice path (a 256-cell tile made of four
 * 4 x 4 x 4 bricks of one Cartesian grid), then resets both.  Synchronises
 * the device.  GRF_EINVAL for NULL pointers, GRF_ECUDA if unreadable.
 */
int grf_take_adjoint_path_counts(int64_t *general_tiles, int64_t *lattice_tiles);

/*
 * grf_take_grid_tiles -- tiles of 128 x 128 cells computed by the tensor-core
 * grid path since the last call, then resets the count.  Synchronises the
 * device.  GRF_EINVAL for NULL, GRF_ECUDA if the counter cannot be read.
 */
int grf_take_grid_tiles(int64_t *tiles);

/*
 * grf_take_grid_adjoint_units -- units (128 modes x 64 x cells x 64 (y, z)
 * cells) computed by the tensor-core grid adjoint since the last call, then
 * resets the count.  Synchronises the device.  GRF_EINVAL for NULL,
 * GRF_ECUDA if the counter cannot be read.
 */
int grf_take_grid_adjoint_units(int64_t *units);

/*
 * grf_debug_grid_path -- process-wide setting of the grid path (enable = 0:
 * grid plans take the CUDA-core paths, for comparisons; 1, the default, and
 * 2: every grid plan takes the grid path, forward and adjoint; grids of at
 * most 64 tiles of 128 x 128 cells split each tile's modes over several
 * CTAs) and the number of
 * 32-mode chunks the tensor-core accumulator sums before each fold into the
 * running sum (fold_chunks = 1, 2, 4 or 8, lowered to a divisor of the
 * table's chunk count; default 4).  GRF_EINVAL otherwise.
 */
int grf_debug_grid_path(int32_t enable, int32_t fold_chunks);

/*
 * grf_debug_mma_f16 -- self-test of the tensor-core path's operand layout,
 * descriptors and accumulator read-back:
 * D[r][c] = sum_k A[r][k] B[c][k] for r, c < 128 and k < 64 k_chunks, with
 * A and B device arrays of 128 x (64 k_chunks) FP16 bit patterns (rows
 * contiguous) and D a device array of 128 x 128 floats (row-major), summed in
 * chunks of 64 into one FP32 accumulator.  status_dev: device int32 that gets
 * bit 2 if a bounded wait expired.  GRF_EINVAL for NULL pointers or k_chunks
 * outside [1, 4096].  Asynchronous on `stream`.
 */
int grf_debug_mma_f16(const uint16_t *A, const uint16_t *B, int32_t k_chunks, float *D, int32_t *status_dev,
                      void *stream);

/*
 * grf_debug_inject_alloc_failures -- host-side fault injection for tests
 * (the paper has no counterpart).  The next n host allocations made by the
 * library's entry points fail as if the allocator had run out of memory: the
 * entry point that meets one returns GRF_ENOMEM with grf_last_error() set,
 * launches nothing after that point and leaves earlier plans, tables and
 * batches usable.  n = 0 clears the injection.  Every entry point catches
 * host exceptions, so none crosses this ABI.  Returns GRF_EINVAL for n < 0.
 */
int grf_debug_inject_alloc_failures(int32_t n);

/*
 * grf_mufu_probe -- throughput probe of the hardware cosine: `iters`
 * dependent-free cos.approx evaluations per thread over a grid of
 * `blocks` x 256 threads; writes one float per thread to `sink` (device,
 * blocks * 256 floats) so nothing is optimised away.
 */
int grf_mufu_probe(int32_t blocks, int32_t iters, float *sink, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GRF_H */
