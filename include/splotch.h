/*
 * splotch.h -- C ABI of the GB300 (sm_103a) Splotch frame renderer.
 *
 * The library renders one frame of a particle set the way Sec. 2 of
 * "GPU Accelerated Particle Visualization with Splotch" (Rivi et al.)
 * describes it: rasterisation (normalisation, roto-translation and
 * perspective projection, colour look-up, activity test) followed by the
 * rendering of every active particle as the clipped Gaussian of Eq. 2,
 * accumulated additively (Eq. 1 with E_p = A_p, so the order of particles
 * does not matter).  Particles are classified by their screen radius
 * (Eq. 7) as in Sec. 4: point-like (r <= r_sml), tile-resident and large.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: SPL_OK (0) or one of the SPL_E*
 *     codes below; spl_error_string() names it.  No C++ exception crosses
 *     the boundary.
 *   - Invalid arguments return SPL_EINVAL and change nothing.  Allocation
 *     failure returns SPL_ENOMEM.  A CUDA error raised by an earlier,
 *     asynchronous launch is returned by the next call that synchronises
 *     (SPL_ECUDA); a device-side check that failed (a list overflow or an
 *     index guard) is returned as SPL_EDEVICE by the next render call (the
 *     flag is then cleared).
 *   - One context belongs to one device and one CUDA stream; it is not
 *     thread-safe.  All device work of a call is issued on the context's
 *     stream unless the call takes a stream argument, in which case that
 *     stream is used.  NULL means the legacy default stream.
 *   - Pointers marked "device" must be device memory of the context's
 *     device (for example a torch CUDA tensor's data_ptr()); pointers marked
 *     "host" are ordinary (preferably pinned) host memory.
 *   - The library owns the particle storage and all scratch memory; the
 *     caller owns images and every buffer it passes in.
 *   - Images are row-major, y downwards, RGB interleaved, FP32:
 *     pixel (i, j) channel c lives at index 3 * (j * width + i) + c.
 */
#ifndef SPLOTCH_H
#define SPLOTCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SPL_OK 0
#define SPL_EINVAL 1    /* invalid argument */
#define SPL_ENOMEM 2    /* device or host allocation failed */
#define SPL_ECUDA 3     /* CUDA runtime error */
#define SPL_ESTATE 4    /* call out of order (e.g. render before particles) */
#define SPL_EDEVICE 5   /* a device-side check failed during the last render */
#define SPL_ELIMIT 6    /* a size beyond the fixed scratch of spl_render_noalloc */

/* memory space of caller buffers */
#define SPL_MEM_HOST 0
#define SPL_MEM_DEVICE 1

/* storage type of the per-particle attributes h, I, s */
#define SPL_ATTR_F32 0    /* h, I, s in FP32: 24 B per particle */
#define SPL_ATTR_F16 1    /* h, I, s in IEEE binary16, widened to FP32 on load: 18 B per
                             particle (the memory-access model of Sec. 3.2: one load per
                             particle, fewer bytes).  h enters exp(-d^2/h^2), so its 2^-11
                             rounding moves clip-edge weights by up to ~1e-2 relative: this
                             layout does NOT keep images within 2e-3 of the FP32 originals
                             (measured 2.5e-3); the next two layouts do */
#define SPL_ATTR_F16_IS 2 /* h in FP32, I and s in binary16: 20 B per particle; images
                             within 2e-3 of the FP32 originals (measured 9e-4) */
#define SPL_ATTR_LOGH16 3 /* I and s in binary16, h as a 16-bit logarithmic code k (uint16):
                             h = 2^(h_log2_min + k / 4096), 1/4096-octave steps over 16
                             octaves (relative step 1.7e-4, a third of binary16's): 18 B per
                             particle, images within 2e-3 of the FP32 originals (measured
                             1.3e-3); spl_load_particles_as / spl_encode_attrs write it */

/* output modes */
#define SPL_MODE_ADDITIVE 0   /* image = sum of clipped Gaussians (Eq. 1, E_p = A_p, thin) */
#define SPL_MODE_EA 1         /* image = 1 - exp(-sum), the E_p = A_p solution of Eq. 1 */
#define SPL_MODE_ABSORB 2     /* Eq. 1 with E_p != A_p over depth-ordered particles: emission
                               * E_p = brightness I_p colour(s_p), grey absorption
                               * A_p = absorption * brightness * I_p; across particle p a ray
                               * becomes I exp(-tau) + (E_p/A_p)(1 - exp(-tau)), tau = A_p w_p,
                               * particles crossed from the farthest to the nearest, equal
                               * depths by decreasing particle index.  The depth key is z_c
                               * rounded to FP32, so particles whose depths lie within one FP32
                               * ulp of each other are ordered by index.  Single views only
                               * (spl_render, spl_render_host) */

/* tile schedulers */
#define SPL_SCHED_NONE 0      /* tiles in image order */
#define SPL_SCHED_COUNT 1     /* longest-first by the count heuristic */
#define SPL_SCHED_MLP 2       /* longest-first by the tile-cost network */

typedef struct spl_ctx spl_ctx;

/* Particle set (Sec. 2 "Data Loading": at least three coordinates, plus the
 * smoothing length, an intensity and a colour scalar).  n may be 0. */
typedef struct {
    int64_t n;
    const float *x, *y, *z;    /* positions, FP32, n each */
    const void *h, *I, *s;     /* smoothing length, intensity, colour scalar:
                                  float or binary16 according to attr_type */
    int32_t attr_type;         /* SPL_ATTR_F32, SPL_ATTR_F16, SPL_ATTR_F16_IS or SPL_ATTR_LOGH16 */
    int32_t mem_space;         /* SPL_MEM_HOST or SPL_MEM_DEVICE (all arrays) */
    const float *cr, *cg, *cb; /* optional colour components (FP32, n each, all three or none):
                                  they replace the palette look-up, e = brightness * I * (c_R,
                                  c_G, c_B) -- the vector quantities of Sec. 2 (e.g. a velocity
                                  gives R, G, B); a non-finite component makes the particle
                                  inactive */
    float h_log2_min;          /* SPL_ATTR_LOGH16: log2 of the smoothing length of code 0 (finite) */
} spl_particles;

/* Pinhole camera (Sec. 2 "roto-translated and projected according to camera
 * settings").  Basis: fwd = unit(target - eye), right = unit(fwd x up),
 * up' = right x fwd; focal length f = (height/2) / tan(fov_y/2);
 * x_s = width/2 + f x_c / z_c, y_s = height/2 - f y_c / z_c; pixel (i, j)
 * has its centre at (i + 1/2, j + 1/2).  Particles with z_c <= z_near are
 * inactive. */
typedef struct {
    double eye[3], target[3], up[3];
    double fov_y_deg;          /* in (0, 180) */
    int32_t width, height;     /* 1 .. 16384 */
    double z_near;             /* > 0 */
} spl_camera;

/* Render parameters.  Eq. 2: rho = rho0 exp(-d^2/sigma^2), clipped beyond
 * chi*sigma; sigma = sigma_per_h * h; Eq. 7: r = chi * sigma * f / (z_c s_box).
 * r_sml is the point-rule radius of Sec. 4; r_small and r_large only choose
 * how a particle is processed (they never change the image). */
typedef struct {
    double chi;                /* clip factor (default 3) */
    double sigma_per_h;        /* default 1 */
    double s_box;              /* S_box of Eq. 7 (default 1) */
    double r_sml;              /* point rule for r <= r_sml (default 0.5) */
    double brightness;         /* emission scale (default 1) */
    int32_t tile_px;           /* tile side t_x = t_y of Eq. 8: 16, 32 or 64 (default 32) */
    double r_small;            /* r_sml < r <= r_small: one thread per particle over its pixel box
                                * (default 2; r_small = r_sml: no such class) */
    double r_large;            /* r > r_large: large pass (default 64) */
    int32_t mode;              /* SPL_MODE_ADDITIVE, SPL_MODE_EA or SPL_MODE_ABSORB */
    int32_t sched;             /* SPL_SCHED_* (default SPL_SCHED_NONE) */
    double absorption;         /* SPL_MODE_ABSORB: A_p = absorption * brightness * I_p, > 0 (default 1) */
    int32_t log_flags;         /* SPL_LOG_I | SPL_LOG_S (default 0): logarithms of processed
                                  quantities (Sec. 2) */
} spl_params;

/* log_flags: I is replaced by log10(I); s is replaced by log10(s) before its
 * normalisation (s_min and s_max of the colour map are then in log units).  A
 * non-positive value under a logarithm makes the particle inactive. */
#define SPL_LOG_I 1
#define SPL_LOG_S 2

/* Per-frame statistics of the last render (counts are exact).  With timing
 * enabled (spl_set_timing) every render records CUDA events between its
 * stages on the render stream; the ms_* fields are the last frame's stage
 * times and sum_ms[] / timed_frames accumulate them (order: raster, bin,
 * tile, large, epilogue, total) since timing was last enabled.  Reading the
 * stats waits for the last frame to finish. */
typedef struct {
    int64_t n_particles, n_active, n_point, n_small, n_medium, n_large;
    int64_t n_entries[4];      /* tile-list entries: point, small, medium, large */
    int32_t n_tiles, tile_px;
    float ms_raster, ms_bin, ms_tile, ms_large, ms_epilogue, ms_total;
    int64_t timed_frames;
    double sum_ms[6];
    int32_t launches;          /* kernels the last render launched */
} spl_stats;

/* Context lifecycle.  device: CUDA ordinal; stream: cudaStream_t or NULL. */
int spl_create(spl_ctx **out, int device, void *stream);
int spl_destroy(spl_ctx *ctx);     /* NULL is accepted and ignored */

/* Copy a particle set into the library's device SoA storage (replacing any
 * earlier set).  Host sources are copied with cudaMemcpyAsync on the
 * context stream; the call returns after the copy has completed. */
int spl_load_particles(spl_ctx *ctx, const spl_particles *p);

/* Load FP32 attributes and store them in a smaller layout (the memory-access
 * model of Sec. 3.2: every particle's bytes are read once per frame, so fewer
 * bytes per particle is less traffic).  p->attr_type must be SPL_ATTR_F32;
 * store_as is SPL_ATTR_F32, SPL_ATTR_F16, SPL_ATTR_F16_IS or SPL_ATTR_LOGH16
 * (then h_log2_min, finite, is the log2 of the smoothing length of code 0).
 * The conversion runs on the device (spl_encode_attrs); host arrays are first
 * copied into temporary device memory.  Otherwise as spl_load_particles. */
int spl_load_particles_as(spl_ctx *ctx, const spl_particles *p, int32_t store_as,
                          float h_log2_min);

/* Convert n FP32 attributes (d_h, d_I, d_s: DEVICE, of ctx's device) into the
 * storage layout store_as, written to d_h_out, d_I_out, d_s_out (DEVICE,
 * caller-owned; 4 bytes per value where the layout keeps FP32, 2 bytes for
 * binary16 and for the h code).  Binary16 values are rounded to nearest even.
 * SPL_ATTR_LOGH16 codes are k = round_half_even(4096 (log2 h - h_log2_min))
 * clamped to [0, 65535], formed in FP64; h = 0 gets code 0; a negative or
 * non-finite h (a particle the FP32 layout renders inactive) gets code 0 and
 * its I is stored as a binary16 NaN, which keeps the particle inactive.
 * stream: NULL means the context stream; returns with the kernel queued. */
int spl_encode_attrs(spl_ctx *ctx, const float *d_h, const float *d_I, const float *d_s,
                     int64_t n, int32_t store_as, float h_log2_min, void *d_h_out,
                     void *d_I_out, void *d_s_out, void *stream);

/* Camera, colour map and parameters.  The colour map is n >= 1 RGB FP32
 * triples (host memory), looked up by s' = clamp((s - s_min)/(s_max - s_min),
 * 0, 1) with linear interpolation between the n entries (Sec. 2 palettes). */
int spl_set_camera(spl_ctx *ctx, const spl_camera *cam);
int spl_set_colormap(spl_ctx *ctx, const float *rgb, int32_t n, float s_min, float s_max);  /* 1 <= n <= 1024 */
int spl_default_params(spl_params *out);
int spl_set_params(spl_ctx *ctx, const spl_params *q);
int spl_get_params(spl_ctx *ctx, spl_params *out);

/* Render the loaded particles with the current camera into d_image (device,
 * width*height*3 FP32, caller-owned, fully overwritten).  stream: NULL means
 * the context stream.  The call waits once on the host for the binning counts
 * (to size the tile lists); meanwhile the image is cleared and the lists are
 * filled on the device into the capacities of the previous frames, so the
 * device does not drain between binning and the tile pass.  A frame whose
 * lists outgrow those capacities (the first one, or a heavier view) is
 * detected there, the buffers are grown and the lists filled again.  The call
 * returns with the tile and large passes queued on the stream. */
int spl_render(spl_ctx *ctx, float *d_image, void *stream);

/* Same, into host memory: renders into library scratch and copies the image
 * to h_image (width*height*3 floats); returns when the copy has completed. */
int spl_render_host(spl_ctx *ctx, float *h_image);

/* Out-of-core render (Sec. 3.2, Eq. 3: a data set larger than device memory
 * is split into chunks that pass through the device one after the other).
 * p: particles in HOST memory (p->mem_space must be SPL_MEM_HOST; page-locked
 * memory lets the copies overlap the rendering), any count n >= 0, FP32 or
 * FP16 attributes as for spl_load_particles.  chunk >= 1 particles per chunk;
 * the device holds two chunks of attributes at a time (24 B per particle in
 * FP32) plus the per-frame scratch of one chunk.  Chunk k+1 is copied on a
 * second stream while chunk k is rendered on `stream` (NULL: the context
 * stream); every chunk adds its additive image into d_image (device,
 * width*height*3 FP32, caller-owned, overwritten), which is exact because
 * the additive form is linear in the particle set (Sec. 2); the E=A map, if
 * selected, is applied once after the last chunk.  Camera, colour map and
 * parameters are the context's; the particles of spl_load_particles are
 * neither read nor changed.  spl_get_stats then reports the counts summed
 * over the chunks and the last chunk's tile count.  Returns SPL_EINVAL for bad
 * arguments or device-memory particles, SPL_ESTATE without a camera or colour
 * map, SPL_ENOMEM if the chunk buffers do not fit; returns after every copy
 * has completed (the host arrays may be freed), with the last chunk's
 * kernels queued on the stream. */
int spl_render_stream(spl_ctx *ctx, const spl_particles *p, int64_t chunk, float *d_image,
                      void *stream);

/* Render n_views (1 .. 64) cameras of the loaded particle set in one batch;
 * d_images[k] (device) receives cams[k].width * cams[k].height * 3 floats.
 * The particles are rasterised for every view by one launch (each particle
 * is read from HBM once per batch, then hits in L2), the views' tile lists
 * share one scan, and one persistent launch renders every (view, tile) work
 * item, so that light and heavy views balance each other.  The first call
 * for a configuration (number of views, image sizes, parameters, particle
 * count) renders eagerly and then captures the whole pipeline into a CUDA
 * graph; later calls with the same configuration -- the cameras themselves
 * may move -- replay that graph.  A replay whose lists outgrow the captured
 * capacities is detected on the device and the batch is rendered again
 * eagerly.  Returns after the batch has finished. */
int spl_render_batch(spl_ctx *ctx, const spl_camera *cams, int32_t n_views,
                     float *const *d_images, void *stream);

/* Autotuner (the empirical tuning of tile size and chunking of Sec. 5.1,
 * done by timing): renders the batch with every candidate tile side
 * (16, 32, 64) and class-radius pair (r_small, r_large) in {(2, 32), (2, 64),
 * (2, 128), (2, inf), (3, 64), (r_sml, 64)}, reps timed renders each, keeps the fastest as the
 * context's parameters and returns it in *best (and its time per batch in
 * *best_ms; either may be NULL).  The images are overwritten. */
int spl_autotune(spl_ctx *ctx, const spl_camera *cams, int32_t n_views, float *const *d_images,
                 int32_t reps, spl_params *best, float *best_ms);

int spl_get_stats(spl_ctx *ctx, spl_stats *out);
int spl_set_timing(spl_ctx *ctx, int32_t enable);   /* per-stage CUDA events; resets sums */

/* enable (default) or disable the CUDA-graph replay of spl_render_batch; with
 * graphs disabled every batch renders eagerly, with per-stage timing. */
int spl_set_graph(spl_ctx *ctx, int32_t enable);

/* Work of the current camera and particle set, counted exactly by a separate
 * diagnostic kernel (not part of a render): out[0] = point deposits that land
 * on the image, out[1..3] = covered (particle, pixel) pairs, d^2 <= r^2, of
 * the small, medium and large classes.  Used for roofline accounting. */
int spl_count_work(spl_ctx *ctx, int64_t out[4]);

/* ---- Load balance: learned tile-cost scheduler --------------------------
 * The render's work items (a tile with its lists, or a bounded segment of a
 * crowded tile's list -- Sec. 4 Remarks note how unevenly particles fall into
 * tiles) are taken by persistent CTAs.  With params.sched = SPL_SCHED_COUNT
 * or SPL_SCHED_MLP they are taken longest-first by a predicted cost:
 *   SPL_SCHED_COUNT  heur[0] + heur[1] * log1p(entries of the item);
 *   SPL_SCHED_MLP    the tile-cost network y = w2 . relu(W1 x + b1) + b2,
 *                    32 -> 64 -> 1 in FP32, on the item's 32 features (per
 *                    radius bin b = clamp(floor(log2(r / 0.5)), 0, 15): x[b] =
 *                    log1p(particles in bin b), x[16 + b] = log1p(tile pixels
 *                    inside their boxes / tile area)); without a model it
 *                    falls back to SPL_SCHED_COUNT.
 * Parameter vector (SPL_MLP_NPARAM floats): W1[64][32] row-major, b1[64],
 * w2[64], b2.  The paper has no counterpart to the network. */
#define SPL_MLP_NPARAM 2177

/* Load a model (theta: host, SPL_MLP_NPARAM floats, or NULL to keep) and/or
 * the count heuristic's two coefficients (heur: host, or NULL to keep;
 * default {0, 1}). */
int spl_set_model(spl_ctx *ctx, const float *theta, const float *heur);

/* With recording on, every render also stores each work item's features and
 * the SM clock cycles its CTA spent on it (clock64 difference). */
int spl_set_recording(spl_ctx *ctx, int32_t enable);

/* Copy the last render's samples (at most cap) into DEVICE buffers:
 * d_feat[n][32] features and d_logc[n] = log(cycles).  *n receives the count.
 * Waits for the context stream.  SPL_ESTATE when recording is off. */
int spl_get_samples(spl_ctx *ctx, float *d_feat, float *d_logc, int64_t cap, int64_t *n);

int spl_mlp_nparam(void);   /* SPL_MLP_NPARAM */

/* Network kernels on DEVICE buffers (stream: cudaStream_t or NULL).
 * forward:   d_y[b] = net(d_x[b]) for b < B (d_x row-major [B][32]).
 * loss_grad: d_grad = gradient of L = (1/B) sum_b (net(x_b) - t_b)^2 with
 *            respect to every parameter, d_loss (may be NULL) = L; allocates
 *            and frees its own scratch and waits for the stream.
 * adam:      one Adam step (Kingma & Ba, Algorithm 1) on np parameters,
 *            step >= 1, moments d_m, d_v updated in place. */
int spl_mlp_forward(const float *d_theta, const float *d_x, int64_t B, float *d_y, void *stream);
int spl_mlp_loss_grad(const float *d_theta, const float *d_x, const float *d_t, int64_t B,
                      float *d_grad, float *d_loss, void *stream);
int spl_mlp_adam(float *d_theta, const float *d_grad, float *d_m, float *d_v, int64_t np,
                 int64_t step, float lr, float beta1, float beta2, float eps, void *stream);

/* Full-batch training on the GPU: `steps` Adam steps (beta 0.9 / 0.999,
 * eps 1e-8, learning rate lr) of the mean-squared-error loss on DEVICE
 * samples d_x[B][32], d_t[B], starting from and returning theta (HOST,
 * SPL_MLP_NPARAM floats); losses (HOST, steps floats, may be NULL) receives
 * the loss before each step.  Allocates its own scratch. */
int spl_mlp_train(const float *d_x, const float *d_t, int64_t B, float *theta, int32_t steps,
                  float lr, float *losses, void *stream);

/* The E_p = A_p solution of Eq. 1 applied to an additive image: every one of
 * the n_values floats v of d_image (DEVICE, of ctx's device) becomes
 * 1 - exp(-v), in place (the map is not linear, so a frame composed from
 * partial additive images -- the particle chunks of Sec. 2's MPI scheme, or
 * out-of-core chunks -- takes it once, after the sum).  stream: NULL means the
 * context stream; returns with the kernel queued. */
int spl_apply_ea(spl_ctx *ctx, float *d_image, int64_t n_values, void *stream);

/* Diagnostics used by the tests.  spl_get_records copies the last render's
 * per-particle rasterisation results for particles [0, n) into host arrays
 * (any may be NULL): screen position x_s, y_s (as double), screen radius r,
 * emission e (n*3), class (-2 inactive, 0 point, 1 small, 2 medium, 3 large). */
int spl_get_records(spl_ctx *ctx, int64_t n, double *xs, double *ys, float *r,
                    float *e, int32_t *cls);

/* Render without allocating: for callers that cannot let a library call
 * cudaMalloc -- an application whose device memory is handed out by its own
 * allocator or held to a fixed budget, or a host program that passes only its
 * own buffers and wants no hidden device allocation.  It needs no context.  It
 * runs the kernels of spl_render, with every scratch buffer carved from one
 * file-scope __device__ array of about 16 MiB, which every GPU that
 * loads the library holds until the process exits.  The paper has no
 * counterpart: it is a property of this library, not of the method.
 *   p       particles in DEVICE memory (mem_space must be SPL_MEM_DEVICE),
 *           n <= 131072;
 *   cam     camera with ceil(width/tile) * ceil(height/tile) <= 16384 tiles;
 *   q       parameters, or NULL for spl_default_params(); q->sched is ignored
 *           (work items are taken in image order), SPL_MODE_ABSORB is rejected;
 *   rgb     colour map (HOST memory, npal RGB triples, 1 <= npal <= 1024)
 *           looked up over [s_min, s_max];
 *   d_image DEVICE output, width*height*3 FP32, fully overwritten;
 *   device  CUDA ordinal; stream: cudaStream_t or NULL.
 * Sizes beyond those limits, or a frame whose tile lists exceed 2^21 entries
 * or 32768 work items, return SPL_ELIMIT and render nothing.  The first call
 * on a device looks up the array's device address (with that device made
 * current).  The call waits on the host once, after binning, for the list
 * sizes, so it must not be issued on a stream that is being captured into a
 * CUDA graph (it then returns SPL_ESTATE without doing anything).  It returns
 * with the tile and large passes queued; a device-side check that fails in
 * those passes (an index guard) is reported as SPL_EDEVICE by the next call on
 * that device, whose own frame is then not rendered.  Every call shares the one
 * array, which keeps the last call's contents (each call clears what must
 * start at zero), so calls whose kernels overlap on the GPU -- on different
 * streams, or from different threads -- race and corrupt each other:
 * serialise them. */
int spl_render_noalloc(const spl_particles *p, const spl_camera *cam, const spl_params *q,
                       const float *rgb, int32_t npal, float s_min, float s_max, float *d_image,
                       int32_t device, void *stream);

const char *spl_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* SPLOTCH_H */
