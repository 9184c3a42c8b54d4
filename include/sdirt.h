/*
 * sdirt.h -- C ABI of the GB300 (sm_103a) dual-pixel (DP) simulator hot path.
 *
 * Method: He et al., "Simulating Dual-Pixel Images From Ray Tracing For Depth
 * Estimation" (ICCV 2025).  The library computes
 *   1. a sequential real-ray trace of a lens from an object point through N x N
 *      entrance-pupil samples (Sec. 3.1),
 *   2. the left/right DP sub-pixel decision of every sensor hit (Sec. 3.1,
 *      Eq. 1 inside the microlens, Eq. 2 outside) and the DP PSF pair
 *      accumulated from unit ray energies (Eq. 3), sum-normalised (Sec. 3.2),
 *   3. per-pixel rendering of the left/right DP images from an all-in-focus
 *      image and a depth map with each pixel's own flipped DP PSF on the
 *      replicate-padded image (supplement, "Local DP PSF convolution"),
 *   and the adjoints of 2 (bilinear splat) and 3.
 *
 * Conventions shared by every call
 *   - Units: mm for lengths, nm for wavelengths, metres for depth maps.
 *     z runs along the optical axis toward the sensor; the vertex of surface 0
 *     is at z = 0; radius > 0 puts the centre of curvature at +z.
 *   - Ownership: the caller owns every device buffer and the stream.  The
 *     library owns only the opaque sd_lens (a host struct plus one slot of a
 *     __constant__ lens table on each device it was uploaded to).  No call
 *     allocates device memory except sd_lens_load, which allocates none either
 *     (constant memory is static); hot calls never allocate.
 *   - Errors: every function returns sd_status.  Argument errors are reported
 *     synchronously before anything is launched.  SD_ERR_CUDA wraps a failed
 *     CUDA runtime call (the CUDA error is kept in sd_last_cuda_error()).
 *     Ray-level failures (vignetting, TIR, no intersection, Newton
 *     non-convergence) are statistics, not errors.
 *   - Streams: every device call is asynchronous on the given stream
 *     (0 = legacy default stream).
 *   - Thread safety: calls on distinct lenses and streams may run
 *     concurrently; sd_lens_load/sd_lens_free serialise on a library mutex.
 */
#ifndef SDIRT_H
#define SDIRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int sd_status;
enum {
  SD_OK = 0,
  SD_ERR_ARG = 1,          /* null pointer, size out of range, bad enum */
  SD_ERR_LENS = 2,         /* invalid prescription (see sd_lens_load) */
  SD_ERR_UNSUPPORTED = 3,  /* valid but not supported (e.g. ks > 127) */
  SD_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  SD_ERR_CAPACITY = 5,     /* library table full (lens slots), or a fixed
                              device array too small for the sizes */
  SD_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up (reported by
                              sd_sync_status from a status word) */
};

/* ------------------------------------------------------------------------
 * Lens (Sec. 3.1 lens model; Tables S1/S2 columns)
 * ---------------------------------------------------------------------- */
enum { SD_SURF_REFRACT = 0, SD_SURF_STOP = 1 };
#define SD_MAX_SURFACES 32
#define SD_MAX_LENSES 16

typedef struct sd_surface {
  int32_t type;          /* SD_SURF_REFRACT or SD_SURF_STOP (flat aperture) */
  int32_t reserved;
  double radius;         /* mm; 0 = flat */
  double thickness;      /* mm to the next surface; last: to the sensor */
  double nd, vd;         /* medium after the surface; nd = 1 is air; vd <= 0
                            means non-dispersive (n = nd at every wavelength) */
  double semi_diameter;  /* clear aperture radius, mm (stop radius for a stop) */
  double conic;          /* k */
  double asph[5];        /* a4, a6, a8, a10, a12 (sag terms a_2m rho^2m) */
} sd_surface;

typedef struct sd_lens sd_lens; /* opaque */

/* Paraxial (first-order) data of a lens at one wavelength and object depth. */
typedef struct sd_paraxial {
  double efl, bfl;        /* effective and back focal length, mm */
  double z_ep, r_ep;      /* entrance pupil plane z and radius (image of the
                             stop in object space, Sec. 3.1) */
  double sensor_dist;     /* last surface vertex -> sensor, mm */
  double m_sensor;        /* paraxial chief-ray height on the sensor per unit
                             object height at this depth */
  double img_dist;        /* paraxial image distance after the last vertex */
  double z_sensor;        /* sensor plane z */
} sd_paraxial;

/*
 * Validates a prescription of n (<= SD_MAX_SURFACES) surfaces, exactly one of
 * them SD_SURF_STOP, and uploads it to a slot of the device lens table of the
 * current CUDA device.  When focus_mm > 0 the last thickness is replaced by
 * the paraxial image distance (587.5618 nm) of an axial object focus_mm in
 * front of surface 0, i.e. the sensor is put in focus for that depth.
 * Validation: finite numbers, nd >= 1, semi_diameter > 0, no aperture larger
 * than its sphere (1 - (1+k) c^2 sd^2 >= 0), positive thickness except between
 * a stop and its neighbour, positive sensor distance.
 * Returns SD_ERR_LENS on a bad prescription, SD_ERR_CAPACITY when all
 * SD_MAX_LENSES slots are in use.  *out is owned by the caller and released
 * by sd_lens_free.  Host call; synchronous (cudaMemcpyToSymbol).
 */
sd_status sd_lens_load(const sd_surface* surfs, int n, double focus_mm,
                       sd_lens** out);

/* Paraxial data (FP64, host) at lambda_nm for an object at depth_mm. */
sd_status sd_lens_paraxial(const sd_lens* lens, double lambda_nm,
                           double depth_mm, sd_paraxial* out);

/* Changes one lens parameter and re-uploads the device image.  Parameter
 * id = surface*8 + j with j = 0 curvature (1/mm), 1 conic, 2..6 a4..a12,
 * 7 thickness after the surface (the last surface's thickness is the sensor
 * distance).  Later traces compute ray generation (object point, entrance
 * pupil) from the changed lens.  Host call; synchronous. */
sd_status sd_lens_set_param(sd_lens* lens, int param_id, double value);

sd_status sd_lens_free(sd_lens* lens);

/* ------------------------------------------------------------------------
 * DP sensor (Sec. 3.1: microlens radius r, focal length f, sub-pixel to
 * microlens distance h, sub-pixel width w, pixel pitch ps; Eq. S1 gives
 * h = 0.78 ps, f = 1.44 ps, w = 0.30 ps, r = 0.50 ps).  All in mm; f > h.
 * ---------------------------------------------------------------------- */
typedef struct sd_dp_sensor {
  double pitch_mm, h_mm, f_mm, w_mm, r_mm;
} sd_dp_sensor;

/* ------------------------------------------------------------------------
 * PSF requests.  One request = one object point p (Sec. 3.1): (h_mm, v_mm)
 * is the point of the sensor plane (x, y, relative to the optical axis) at
 * which the paraxial chief ray lands; the object sits at depth_mm in front of
 * surface 0 at the object point that makes this so (a radial bank uses
 * v_mm = 0; a per-pixel PSF map uses every pixel's 2-D position).  Rays:
 * N x N cell-centred samples on the entrance-pupil square kept inside the
 * pupil disc (exactly: (2i+1-N)^2 + (2j+1-N)^2 <= N^2).  The PSF patch
 * [2][ks][ks] (L plane then R plane, row index along +y, column along +x) is
 * centred on (h_mm, v_mm).
 * ---------------------------------------------------------------------- */
typedef struct sd_psf_request {
  double h_mm;
  double depth_mm;
  double lambda_nm;
  int32_t n_grid;      /* N, 2..2048 */
  int32_t ks;          /* odd, 1..127 */
  int32_t lens;        /* index into the lens array of the call */
  int32_t reserved;
  int64_t out_offset;  /* element offset of this PSF pair in the output */
  double v_mm;         /* image height along y (0 for field points on +x) */
} sd_psf_request;      /* 56 bytes, device-resident */

enum { SD_BIN_HARD = 0, SD_BIN_BILINEAR = 1 };
enum { SD_NORM_NONE = 0, SD_NORM_JOINT = 1, SD_NORM_SEPARATE = 2,
       SD_NORM_PER_RAY = 3 };
enum { SD_F32 = 0, SD_BF16 = 1, SD_F16 = 2 };

typedef struct sd_trace_opts {
  int32_t mode;         /* SD_BIN_HARD (unit impulse into the landing
                           pixel, Eq. 3) or SD_BIN_BILINEAR (unit energy split
                           over the 4 nearest pixel centres; L/R from the
                           landing pixel; differentiable in the lens) */
  int32_t norm;         /* SD_NORM_*: JOINT sum(L+R) = 1 (Sec. 3.2 sum
                           normalisation), SEPARATE each plane sums to 1,
                           PER_RAY divide by the launched ray count */
  int32_t out_dtype;    /* SD_F32, SD_BF16 or SD_F16 */
  int32_t newton_iters; /* asphere Newton iteration cap (0 = 12) */
  int32_t max_ks;       /* required: largest ks of any request (odd, <= 127);
                           sizes the shared-memory patch */
  int32_t max_n_grid;   /* largest N of any request (0 = 512, <= 2048) */
  uint32_t* land_mask;  /* device, nullable: one bit per ray (see
                           sd_dp_psf_trace_mask_bytes).  sd_dp_psf_trace
                           and sd_dp_psf_trace_batched write it;
                           sd_dp_psf_trace_backward reads it and traces
                           again only the rays whose bit is set.  The map
                           and hit-dump entry points ignore it. */
} sd_trace_opts;

/*
 * Bytes of a landing mask for n_req requests with pupil grids up to
 * max_n_grid (0 = 512): request r owns words [r * W, (r + 1) * W), W =
 * ceil(max_n_grid^2 / 32); bit k % 32 of its word k / 32 is ray k of the
 * request (the trace's ray order: in-pupil samples in raster order).
 * sd_dp_psf_trace (and sd_dp_psf_trace_batched, bitwise the same) sets the
 * bit of every ray that reaches the sensor, lands
 * on the L or R sub-pixel (Eq. 1/2) and has its nearest pixel centre at most
 * one pixel outside the request's ks x ks patch (the bilinear footprint of a
 * ray can touch the patch only then), whatever the binning mode, and clears
 * the others; words past a request's ray count are left as they are.  The
 * adjoint takes the same decisions with the same FP32 code, so a ray with a
 * clear bit has no splat gradient there.  A mask holds for the lenses,
 * parameters, sensor and requests it was traced with: an adjoint given a
 * mask takes every ray whose bit is clear to have a zero splat gradient.
 * SD_ERR_ARG for n_req < 0, a null bytes or max_n_grid outside [0, 2048].
 */
sd_status sd_dp_psf_trace_mask_bytes(int n_req, int max_n_grid, size_t* bytes);

/* Per-request statistics (int64 each, device, nullable). */
enum { SD_STAT_LAUNCHED = 0, SD_STAT_REACHED, SD_STAT_L, SD_STAT_R,
       SD_STAT_DP_MISSED, SD_STAT_CLIPPED, SD_STAT_VIGNETTED, SD_STAT_OTHER,
       SD_N_STATS };

/*
 * Traces every request and writes its DP PSF pair at out + out_offset (in
 * elements of out_dtype).  lenses[0..n_lenses) must have been loaded on the
 * current device.  req and stats (n_req x SD_N_STATS int64, nullable) are
 * device pointers; out is device memory large enough for every request.
 * Each PSF is computed by one thread block with a shared-memory patch: no
 * global atomics; results are written exactly once.  Hard mode is exact
 * integer counting (deterministic); bilinear mode accumulates FP32 weights
 * with shared-memory atomics (order-dependent rounding).
 * Stats: launched = reached + vignetted + other; reached = L + R +
 * DP-missed + clipped (a ray whose landing pixel is outside the patch).
 */
sd_status sd_dp_psf_trace(const sd_lens* const* lenses, int n_lenses,
                          const sd_dp_sensor* sensor,
                          const sd_psf_request* req, int n_req,
                          const sd_trace_opts* opts, void* out,
                          int64_t* stats, void* stream);

/*
 * Per-pixel DP PSF map (Sec. 5.1 implementation details; Table S3 times it):
 * one PSF pair for every pixel of an H x W depth map, the object point of
 * pixel (row, col) on the paraxial chief ray through the pixel centre
 * ((col - (W-1)/2) * pitch, (row - (H-1)/2) * pitch) at that pixel's depth
 * (depth_m, device, H x W FP32 metres), one wavelength and one lens.  Writes
 * out (device) as [H][W][2][ks][ks] in opts->out_dtype (the map layout the
 * supplement's render takes) and stats (device, nullable) as
 * [H*W][SD_N_STATS].  The same kernel as sd_dp_psf_trace with the request of
 * each block built on the device; opts->max_ks and max_n_grid are ignored
 * (ks and n_grid size everything).  pitch is the sensor's pixel pitch.
 */
sd_status sd_dp_psf_map(const sd_lens* lens, const sd_dp_sensor* sensor,
                        const float* depth_m, int H, int W, double lambda_nm,
                        int n_grid, int ks, const sd_trace_opts* opts, void* out,
                        int64_t* stats, void* stream);

/*
 * Adjoint of sd_dp_psf_trace in bilinear mode (SD_BIN_BILINEAR) with a
 * linear normalisation (SD_NORM_NONE or SD_NORM_PER_RAY), FP32.  Given
 * grad_out = dLoss/dPSF in the forward's output layout (FP32, out_offset of
 * each request), writes per-request gradients grad_req[r][32*8] with the
 * parameter ids of sd_lens_set_param (surface*8 + {curvature, conic,
 * a4..a12, thickness}; surfaces beyond the lens are zero) and, if grad_lens
 * is not null, their sum per lens grad_lens[l][32*8] (requests summed in
 * index order: deterministic).  Each ray is traced again (nothing is stored
 * between the passes) and swept backward through the sensor propagation,
 * Snell's law, the normal and the intersection (implicit-function
 * derivative at the converged Newton root); ray generation and the discrete
 * decisions (reached, side, splat pixel) are held fixed.  A request whose
 * grad_out patch is all zero has a zero gradient and traces no ray.  The paper trains
 * no lens; this is the differentiable form of Sec. 3.1 / Eq. 3.
 * grad_req and grad_lens are device memory owned by the caller.
 * swept (device, nullable) receives per request [n_req][2] int64: the rays
 * whose splat gradient is non-zero (the rays whose reverse sweep carries a
 * contribution) and the ray slots that ran the sweep (64 per warp in which
 * any ray has a contribution: each thread sweeps two rays as a pair); the
 * first is the adjoint's algorithmic work, the second what the hardware
 * executed.
 * With opts->land_mask (written by sd_dp_psf_trace or sd_dp_psf_trace_batched
 * of the same lenses, sensor, requests and max_n_grid) only the rays whose
 * bit is set are traced
 * again, taken in ray order from a queue that keeps every warp but the
 * request's last full: the gradient equals the maskless one up to the order
 * of FP32 additions (deterministic either way).
 */
sd_status sd_dp_psf_trace_backward(const sd_lens* const* lenses, int n_lenses,
                                   const sd_dp_sensor* sensor,
                                   const sd_psf_request* req, int n_req,
                                   const sd_trace_opts* opts,
                                   const float* grad_out, float* grad_req,
                                   float* grad_lens, int64_t* swept, void* stream);

/*
 * Batched trace of uneven requests (different N, ks, wavelength, lens) in one
 * persistent launch: hard binning only, results identical to
 * sd_dp_psf_trace.  A preparation pass splits every request into work items
 * of whole pupil rows (about rays_per_item rays each); a fixed grid of
 * blocks_per_sm blocks per SM processes contiguous, equal ranges of items,
 * accumulating in a shared-memory patch while consecutive items belong to
 * one request and adding it to the request's u32 counts with integer
 * atomics (order-independent, so deterministic); the block that completes a
 * request normalises and stores it.  No host synchronisation and no
 * allocation: the call can be captured in a CUDA graph.  total_elems is the
 * size of out (every request's out_offset + 2 ks^2 must fit); the workspace
 * (sd_dp_psf_trace_batched_workspace bytes) is device memory of the caller.
 */
typedef struct sd_batch_config {
  int32_t threads;        /* threads per block, multiple of 32 in 64..1024 (0 = 512) */
  int32_t rays_per_item;  /* target rays per work item (0 = 16384) */
  int32_t blocks_per_sm;  /* persistent blocks per SM (0 = 1) */
  int32_t reserved;
} sd_batch_config;

sd_status sd_dp_psf_trace_batched_workspace(int n_req, long long total_elems,
                                            size_t* bytes);

sd_status sd_dp_psf_trace_batched(const sd_lens* const* lenses, int n_lenses,
                                  const sd_dp_sensor* sensor,
                                  const sd_psf_request* req, int n_req,
                                  const sd_trace_opts* opts,
                                  const sd_batch_config* cfg, void* out,
                                  long long total_elems, int64_t* stats,
                                  void* workspace, size_t workspace_bytes,
                                  void* stream);

/*
 * Autotuner of sd_dp_psf_trace_batched: times every candidate configuration
 * (threads 256/512/1024 x rays per item 4096..65536 x 1-2 blocks per SM,
 * within the shared-memory and thread limits) on the caller's batch with
 * CUDA events (one warm-up run, median of three) and returns the fastest in
 * *best.  When cache_path is not null, a previous result for the same key
 * (device name, SM count, n_req, total_elems, max_ks, max_n_grid, n_lenses)
 * is returned from that text file without timing, and new results are
 * appended to it.  Synchronises the stream; writes out and stats.
 */
sd_status sd_dp_psf_trace_batched_tune(const sd_lens* const* lenses,
                                       int n_lenses, const sd_dp_sensor* sensor,
                                       const sd_psf_request* req, int n_req,
                                       const sd_trace_opts* opts, void* out,
                                       long long total_elems, int64_t* stats,
                                       void* workspace, size_t workspace_bytes,
                                       void* stream, const char* cache_path,
                                       sd_batch_config* best);

/*
 * Per-ray record of one request (test and debugging aid): for the k-th
 * in-pupil ray in raster order (pupil row major), rec[k*8 ..] = x, y, dx, dy,
 * dz (landing point and unit direction, FP32), state (0 reached, 1 no
 * intersection, 2 clipped by an aperture, 3 TIR, 4 Newton failed,
 * 5 backwards), side (0 L, 1 R, 2 DP-missed), packed pixel (b * 65536 + a,
 * or -1 outside the patch) -- the last three as floats.  rec is device
 * memory of max_rays * 8 floats; n_rays (device int32) receives the count.
 */
sd_status sd_dp_trace_hits(const sd_lens* lens, const sd_dp_sensor* sensor,
                           const sd_psf_request* req_host,
                           const sd_trace_opts* opts, float* rec,
                           int max_rays, int32_t* n_rays, void* stream);

/* ------------------------------------------------------------------------
 * Rendering (supplement, "Local DP PSF convolution")
 *   out_L[n,c,y,x] = sum_{i,j} Ipad[n,c,y+i,x+j] K_L(y,x,c)[ks-1-i][ks-1-j]
 * with Ipad the image replicate-padded by p = (ks-1)/2, likewise R, output
 * channels [L(0..C-1), R(0..C-1)] (N, 2C, H, W).
 * Bank mode: K(y,x,c) = (1-t) B[f][z0][l] + t B[f][z0+1][l] with l = c when
 * the bank holds C wavelengths (else 0), f the field height nearest to the
 * pixel's radial image height rho = |((x,y) - ((W-1)/2,(H-1)/2)) * pitch|,
 * (z0, t) the bracket of the pixel depth linear in inverse depth, clamped
 * to the first/last slice.  This selection is computed in FP32 without
 * contraction: X = ((float)x - 0.5f*(W-1)) * pitch, rho = sqrtf(X*X + Y*Y),
 * q = 1.0f / depth, iq_j = 1.0f / depths_m[j].
 *
 * Quadrant mode (field_mode = SD_FIELD_QUADRANT): the bank holds a 2-D grid
 * of field points of the first quadrant, [Fx = F][Fy = F][Z][NL][2][ks][ks]
 * with both axes sampled at field_h_mm (>= 0).  A pixel takes the grid point
 * nearest to (|X|, |Y|) on each axis separately (same rule as the radial
 * lookup), and the flip symmetry of the DP PSF about both axes (Sec. 5.3):
 * X < 0 mirrors the kernel's columns and exchanges L and R (the DP split is
 * along x), Y < 0 mirrors its rows.  Removes the radial approximation of
 * off-axis azimuths.  All render entry points take it: sd_dp_render_tc's
 * workspace then holds the four flip classes, and the backward's bank
 * gradient goes through one gradient slab per key (flip class) in its
 * workspace, folded onto the stored quadrant in a fixed order.
 * ---------------------------------------------------------------------- */
#define SD_MAX_BANK_FIELDS 256
#define SD_MAX_BANK_DEPTHS 256
#define SD_FIELD_RADIAL 0
#define SD_FIELD_QUADRANT 1

typedef struct sd_bank_layout {
  int32_t n_field, n_depth, n_lambda, ks;   /* bank [F][Z][NL][2][ks][ks] */
  int32_t dtype;                            /* SD_F32 / SD_BF16 / SD_F16 */
  int32_t field_mode;                       /* SD_FIELD_RADIAL (0) or
                                               SD_FIELD_QUADRANT: bank
                                               [F][F][Z][NL][2][ks][ks] */
  const float* field_h_mm;  /* host, F ascending field heights (mm) */
  const float* depths_m;    /* host, Z ascending depths (m) */
  float pitch_mm;           /* sensor pixel pitch of the rendered image */
  float reserved2;
} sd_bank_layout;
/*
 * Every call that takes a layout validates it on the host before any CUDA
 * call: SD_ERR_ARG for a null layout or height/depth array, n_field outside
 * 1..SD_MAX_BANK_FIELDS, n_depth outside 1..SD_MAX_BANK_DEPTHS, n_lambda < 1,
 * ks < 1 or even, pitch_mm <= 0 (or NaN), field heights or depths not
 * strictly ascending, a depth <= 0, a field_mode other than the two above,
 * or a quadrant bank whose first height is negative; SD_ERR_UNSUPPORTED for
 * ks > 127.
 */

/*
 * aif (N,C,H,W) and out (N,2C,H,W) in image_dtype (SD_F32 / SD_BF16 /
 * SD_F16); depth_m (N,H,W) FP32; bank in layout->dtype.  All device, dense,
 * 16-byte aligned.  Accumulation is FP32.  C must equal n_lambda or
 * n_lambda must be 1.  Deterministic (no atomics across blocks).
 */
sd_status sd_dp_render(const void* aif, const float* depth_m, const void* bank,
                       const sd_bank_layout* layout, int N, int C, int H,
                       int W, int image_dtype, void* out, void* stream);

/*
 * Render from a per-pixel PSF map (supplement, "Local DP PSF convolution":
 * the listing's form, one kernel pair per pixel shared by all channels):
 *   out_L[n,c,y,x] = sum_{u,v} Ipad[n,c,y+u,x+v] map[y][x][0][ks-1-u][ks-1-v]
 * (R with plane 1), Ipad replicate-padded by (ks-1)/2.  aif (N,C,H,W) and out
 * (N,2C,H,W) in image_dtype; psf_map [H][W][2][ks][ks] in map_dtype (the
 * layout sd_dp_psf_map writes); all device.  Accumulation FP32,
 * deterministic.  Storage pairs as sd_dp_render (F32/F32, F32/BF16,
 * BF16/BF16, F16/F16, F32/F16 for image/map); others return
 * SD_ERR_UNSUPPORTED, as do ks > 127.
 * status (device int32, nullable) is zeroed by the call and becomes 1 if a
 * bounded completion wait gave up (out is then invalid; sd_sync_status reads
 * it).  With a status word, ks <= 21, W a multiple of 4 (16-bit map) or 2
 * (FP32 map) and a 16-byte aligned map, the map is streamed into shared
 * memory by bulk copies; otherwise, and always without a status word, it is
 * read with per-thread loads.  Both forms give the same bits.
 */
sd_status sd_dp_render_map(const void* aif, const void* psf_map, int N, int C,
                           int H, int W, int ks, int image_dtype, int map_dtype,
                           void* out, int32_t* status, void* stream);

/*
 * sd_dp_render for 16-bit images on the tensor cores (tcgen05, FP32
 * accumulation in tensor memory): aif (N,C,H,W) and out (N,2C,H,W) in
 * image_dtype (SD_BF16 or SD_F16: both operands of a product share the
 * type), depth_m (N,H,W) FP32, bank in layout->dtype (the image's type, or
 * SD_F32 rounded to it), all device.  Same selection, padding and output
 * layout as sd_dp_render.  Needs a device workspace of
 * sd_dp_render_tc_workspace() bytes, 256-byte aligned (a 16-bit re-layout of
 * the bank written by the call and, in its first word, an error flag set to
 * 1 if a tensor-core completion wait ever gave up; sd_sync_status reads it).
 * Supports ks <= 65 (SD_ERR_UNSUPPORTED otherwise).  Deterministic.
 */
sd_status sd_dp_render_tc(const void* aif, const float* depth_m, const void* bank,
                          const sd_bank_layout* layout, int N, int C, int H,
                          int W, int image_dtype, void* out, void* workspace,
                          size_t workspace_bytes, void* stream);

/* Workspace bytes of sd_dp_render_tc for this bank layout. */
sd_status sd_dp_render_tc_workspace(const sd_bank_layout* layout, size_t* bytes);

/*
 * Adjoint of sd_dp_render (bank mode): given grad_out (N,2C,H,W) FP32 writes
 * grad_aif (N,C,H,W) FP32 and grad_bank (the bank's element layout, FP32),
 * both overwritten; either may be null to skip it.  aif is read in
 * image_dtype and the bank in layout->dtype (the storage types sd_dp_render
 * takes); arithmetic is FP32.  Returns SD_ERR_UNSUPPORTED for another
 * image_dtype.  Both gradients are bitwise reproducible (no atomics on
 * floating-point values; every sum runs in a fixed order).
 * The workspace (device, 256-byte aligned, sd_dp_render_backward_workspace()
 * bytes) holds first the per-pixel slice selection (key and interpolation
 * weight, 8 bytes a pixel, written once and read by both passes), then,
 * when grad_aif is requested, the image pass's tables (the bank re-laid as
 * FP32 kernel columns, each kernel row's non-zero column range), then the
 * bank pass's data.
 *   grad_aif: warps own strips of 64 source columns and 8 output rows; each
 *     scatters its pixels' weighted gradients, slice by slice, into a
 *     warp-private row buffer that is added to the image once; strips whose
 *     footprints overlap run in separate launches in a fixed order.
 *   grad_bank: a thread block per (slice, wavelength) accumulates over the
 *     64x32 tiles that use the slice in a fixed order and writes the slice's
 *     gradient.  A slice with more tiles than a block's share of the launch
 *     is split into two tile chunks while split slots remain: each chunk
 *     block writes a partial slab and the second to finish adds the two in
 *     chunk order.  Blocks start in order of their tile count (the most
 *     first).  Needs the bitmap of the slices each tile uses, for a quadrant
 *     bank a slab of per-flip-class gradients that is then folded, and a
 *     work plan (8 bytes a slice plus the split slots' slabs); split slots
 *     take what the workspace holds beyond that, none if it holds nothing
 *     more (the result then differs from the full workspace's in rounding
 *     only).  Ignored when grad_bank is null.
 * Returns SD_ERR_ARG when a gradient is requested and the workspace is
 * missing, misaligned or smaller than the selection table plus the image
 * tables plus the bitmap (plus the per-key slab of a quadrant bank) plus a
 * work plan without split slots.
 */
sd_status sd_dp_render_backward(const float* grad_out, const void* aif,
                                const float* depth_m, const void* bank,
                                const sd_bank_layout* layout, int N, int C,
                                int H, int W, int image_dtype,
                                float* grad_aif, float* grad_bank,
                                void* workspace, size_t workspace_bytes,
                                void* stream);

/* Device workspace bytes sd_dp_render_backward needs for these sizes (both
 * gradients). */
sd_status sd_dp_render_backward_workspace(const sd_bank_layout* layout, int N,
                                          int C, int H, int W, size_t* bytes);

/*
 * The bank gradient of sd_dp_render_backward on the tensor cores (tcgen05),
 * for 16-bit images: grad_bank (FP32, the stored bank's shape) = the adjoint
 * of the render with respect to the bank, with the image in image_dtype
 * (SD_BF16 or SD_F16), the weighted output gradients w * G rounded to the
 * same type (SD_F16: |w * G| must stay below 65504), products exact and
 * accumulated in FP32 in tensor memory in a fixed order (deterministic).
 * grad_out (N,2C,H,W) FP32, aif (N,C,H,W), depth_m (N,H,W) FP32, all device;
 * the bank itself is not read.  Workspace from
 * sd_dp_render_bank_grad_tc_workspace (device, 256-byte aligned; its first
 * int32 becomes 1 if a bounded completion wait gave up; then the per-pixel
 * slice selection, the tile bitmap, a quadrant bank's per-key slab and the
 * work plan of sd_dp_render_backward's bank pass, whose blocks, slice
 * splits and chunk sums this pass shares).  ks <= 65.  Radial and quadrant
 * banks.
 */
sd_status sd_dp_render_bank_grad_tc_workspace(const sd_bank_layout* layout, int N, int C,
                                              int H, int W, size_t* bytes);
sd_status sd_dp_render_bank_grad_tc(const float* grad_out, const void* aif,
                                    const float* depth_m, const sd_bank_layout* layout,
                                    int N, int C, int H, int W, int image_dtype,
                                    float* grad_bank, void* workspace, size_t workspace_bytes,
                                    void* stream);

/*
 * sd_dp_render_backward for callers that cannot allocate device memory: code
 * that may only use the buffers it is handed (for example a plugin running
 * inside another runtime's memory pool, where a cudaMalloc would bypass the
 * pool or is not permitted).  The paper has no counterpart; this is a
 * deployment variant of the render adjoint with the same arguments minus the
 * workspace and the image dtype (aif is FP32; the bank is read in
 * layout->dtype: FP32, BF16 or FP16).
 * The per-pixel selection table (8 bytes a pixel), the image pass's tables
 * and the bank pass's slice bitmap live in a 16 MiB
 * array that this library reserves statically on every device that loads
 * it (held until the process exits); when what the requested gradients need
 * for these sizes exceeds 16 MiB the call returns SD_ERR_CAPACITY before
 * launching anything.  No device memory is allocated
 * or freed.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: do not use this entry point on a device after cudaDeviceReset
 * (the array then lives at a new address).  Every call uses the same array
 * and it keeps the last call's contents: each call rewrites every word it
 * reads (selection table, re-laid bank, row extents, bitmap), so nothing has
 * to start at zero, but calls that overlap on the GPU (other streams or
 * host threads) race on the array and must be serialised by the caller.
 */
sd_status sd_dp_render_backward_noalloc(const float* grad_out,
                                        const float* aif, const float* depth_m,
                                        const void* bank,
                                        const sd_bank_layout* layout, int N,
                                        int C, int H, int W, float* grad_aif,
                                        float* grad_bank, void* stream);

/*
 * Test aid (the paper has no counterpart): evaluates, on the device, the
 * trace's division and square-root helpers (reciprocal / reciprocal-square-
 * root estimates with one Newton-Raphson correction) on n inputs:
 * quot[i] = a[i] / b[i], root[i] = sqrt(a[i]) (a[i] < 0 is clamped to 0).
 * All arrays device FP32.  Lets a test compare them with correctly rounded
 * IEEE results.
 */
sd_status sd_dev_math_check(const float* a, const float* b, int n, float* quot,
                            float* root, void* stream);

/* ------------------------------------------------------------------------
 * DP PSF prediction network (Sec. 3.2, "Pixel-wise DP image rendering
 * module"; Sec. 5.1 implementation details): an MLP from the normalised object
 * point p = (x_n, y_n, d_n) of a pixel to the 2*ks^2 values of its
 * (PSF_L, PSF_R): 5 hidden layers of 512 neurons (ReLU), a linear output
 * layer of 2*ks^2 neurons; at inference the outputs are clamped at 0 and
 * sum-normalised jointly (sum of L + R = 1).  The paper times this on a
 * 512 x 768 depth map with ks = 21 (0.395 s, supplement table).
 * ---------------------------------------------------------------------- */
#define SD_MLP_HIDDEN 512
#define SD_MLP_MAX_KS 31

/* Bytes of the packed network for kernel size ks (odd, 1..SD_MLP_MAX_KS). */
sd_status sd_mlp_blob_bytes(int ks, size_t* bytes);

/*
 * Packs a network into blob (device memory of sd_mlp_blob_bytes(ks) bytes,
 * 256-byte aligned; owned by the caller).  weights[l] and biases[l], l = 0..5,
 * are host FP32, weights row-major [out][in]: 512x3, four 512x512, and
 * (2 ks^2)x512; biases 512 (l < 5) and 2 ks^2.  The 512-wide matrices are
 * rounded to BF16 (nearest even) and stored in the tensor cores' operand
 * layout; layer 0 and all biases stay FP32.  Synchronous (one host-to-device
 * copy).  SD_ERR_ARG for null pointers, a bad ks or a short blob.
 */
sd_status sd_mlp_pack(const float* const* weights, const float* const* biases, int ks,
                      void* blob, size_t blob_bytes);

/*
 * The DP PSF map of a depth map predicted by the packed network: pixel (y, x)
 * of depth_m (H, W) [metres, FP32, device] has p = (x_n, y_n, d_n) with
 * x_n = (x - (W-1)/2) / (W/2), y_n = (y - (H-1)/2) / (H/2) (the sensor
 * position normalised to [-1, 1]) and d_n = 2 (d - d_min) / (d_max - d_min)
 * - 1; out (H, W, 2, ks, ks) device in out_dtype (SD_F32 or SD_BF16), the
 * layout and dtypes sd_dp_render_map takes.
 * Tensor cores (tcgen05): BF16 operands, FP32 accumulation, hidden
 * activations rounded to BF16 between layers.  *status (device int32) is set
 * to 0 by the call and to 1 by the kernel if one of its bounded completion
 * waits gave up (the map is then invalid).  H * W >= 1, d_max > d_min.
 */
sd_status sd_mlp_psf_map(const void* blob, int ks, const float* depth_m, int H, int W,
                         float d_min_m, float d_max_m, void* out, int out_dtype,
                         int32_t* status, void* stream);

/*
 * Test aid (the paper has no counterpart): runs the tensor-core (tcgen05)
 * path of the BF16 render on a fixed small product, D = A[u:u+128, :] B^T
 * with A (136 x 32) and B (16 x 32) BF16 row-major and D (128 x 16) FP32, all
 * device memory; u in [0, 8] is the row offset applied through the
 * shared-memory descriptor.  *status (device int, zeroed by the caller)
 * becomes 1 if the completion wait timed out.
 */
sd_status sd_dev_tc_check(const void* a, const void* b, int u, float* d,
                          int32_t* status, void* stream);

/* ------------------------------------------------------------------------
 * Device-side status, failure injection and hardware probes (the paper has
 * no counterpart: these serve error reporting, tests and measurement)
 * ---------------------------------------------------------------------- */

/*
 * Waits for the stream and reads a device status word written by a kernel:
 * the first int32 of the workspace of sd_dp_render_tc or
 * sd_dp_render_bank_grad_tc, or the status word of sd_mlp_psf_map or
 * sd_dp_render_map.
 * Returns SD_ERR_TIMEOUT when the word is non-zero (a bounded completion wait
 * of that call gave up: its output is invalid), SD_OK when it is zero,
 * SD_ERR_ARG for a null pointer and SD_ERR_CUDA when the copy fails.
 * Synchronises the stream.
 */
sd_status sd_sync_status(const int32_t* status_word, void* stream);

/*
 * Failure injection for tests: every bounded completion wait (mbarrier poll
 * loop) of the tensor-core kernels and of the bulk-copy map render launched
 * after this call gives up after `polls` polls; polls = 0 makes the first
 * wait of every CTA give up without polling, so that no tensor-core product
 * is issued and the kernel ends through its error path (flag set, the bulk
 * copies already issued waited for, tensor memory freed).
 * polls < 0 restores each kernel's own limit.  Process-wide; host call.
 */
sd_status sd_set_wait_limit(long long polls);

/*
 * FP32 throughput probe: `blocks` blocks of 256 threads, each thread running
 * 16 independent fused multiply-add chains for `iters` iterations
 * (blocks * 256 * iters * 32 flops).  sink (device, blocks * 256 floats) is
 * never written for these arguments; it keeps the arithmetic alive.  Timed
 * by the caller (CUDA events on the stream) to measure the FP32 peak.
 */
sd_status sd_dev_fp32_peak(float* sink, int blocks, int iters, void* stream);

/*
 * Bounds checks of a checked build (the library compiled with -DSD_CHECKED;
 * the paper has no counterpart).  There, the kernels test the indices they
 * compute before the accesses that use them (image and buffer positions,
 * workspace slabs, shared-memory tables, output elements) and skip an access
 * whose index is out of range, recording it.  Synchronises the device, then
 * returns the first failing site (translation unit * 100000 + source line;
 * 0 if none), its index and bound (low 32 bits; index and bound nullable)
 * and the number of failed checks since the last call, and clears the
 * records.  SD_ERR_UNSUPPORTED in the normal build, whose checks compile
 * away; SD_ERR_ARG for a null site or count.
 */
sd_status sd_check_status(int32_t* site, int32_t* index, int32_t* bound, int64_t* count);

/* ------------------------------------------------------------------------
 * Library information
 * ---------------------------------------------------------------------- */
const char* sd_status_string(sd_status s);
/* last CUDA error code seen by the library on this thread (0 if none) */
int sd_last_cuda_error(void);
/* version as 10000*major + 100*minor + patch */
int sd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SDIRT_H */
