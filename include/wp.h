/*
 * wp.h — C ABI of the GB300 (sm_103a) probed adjoint-state gradient library (libwp.so).
 *
 * The library computes, for a batch of independent shots on one GPU, the low-memory
 * imaging method of Louboutin & Herrmann ("Enabling wave-based inversion on GPUs with
 * randomized trace estimation"):
 *   - forward acoustic propagation whose time history is never stored but projected on
 *     the fly onto r probing vectors in time:  Pu = Q^T u_tt           (Eq. 3)
 *   - adjoint propagation projected the same way:  Pv = Q^T v           (Eq. 3)
 *   - the randomized trace estimate of the imaging condition
 *       g[x] = scale * sum_i Pu[i,x] Pv[i,x]                           (Eq. 3, Eq. 1)
 *   - and, as the exact baseline, the full-history (or checkpointed) imaging condition
 *       g = sum_t u_tt[t] v[t]                                          (Eq. 2)
 *
 * Physics (the paper names the isotropic acoustic case, Sec. 2.2, without writing it):
 *   m (u_tt + sigma u_t) - Laplacian(u) = q,  m = 1/v^2 (s^2/m^2),
 * 8th-order central differences in space, 2nd-order leapfrog in time, an absorbing layer
 * of `nbl` cells with damping rate sigma = sigma0 (d/nbl)^2 per axis,
 * sigma0 = 3 damp_v ln(1000) / (2 nbl h), zero values beyond the padded grid.
 * u_tt denotes the m-derivative of the discrete operator at step t (inside the model the
 * centred second difference / dt^2), so that g is exactly dJ/dm of
 * J = 1/2 sum_t |R u[t] - d_obs[t]|^2.
 *
 * Conventions (all calls):
 *   - Grid: interior nx (x), ny (y, 3-D only), nz (z, depth) points padded by nbl cells on
 *     every side: NX = nx + 2 nbl, NY = ny + 2 nbl (1 in 2-D), NZ = nz + 2 nbl,
 *     N = NX*NY*NZ.  Fields are float32 with x fastest: index = (z*NY + y)*NX + x.
 *   - The caller owns every device buffer, the workspace and the stream; the library owns
 *     only the opaque wp_model_t.  Hot calls never allocate device memory: scratch comes
 *     from the caller's workspace, sized by wp_workspace_bytes().
 *   - Every call is asynchronous on the given stream (a cudaStream_t passed as void*;
 *     NULL is the legacy default stream) except wp_model(), which synchronises once to
 *     validate the model.  Every call returns a wp_status; errors never abort the process;
 *     wp_last_error() describes the last failure of the calling host thread.
 *   - Device pointers must be 16-byte aligned.
 *   - Shots are independent: each shot s has its own source/receiver positions and its
 *     own probing matrix Q[s]; batched outputs are shot-major.
 */
#ifndef WP_H
#define WP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WP_OK = 0,
    WP_ERR_INVALID = 1,   /* bad argument: shape, pointer, alignment, position */
    WP_ERR_UNSTABLE = 2,  /* dt violates the leapfrog stability limit of the model */
    WP_ERR_OOM = 3,       /* workspace smaller than wp_workspace_bytes() */
    WP_ERR_CUDA = 4,      /* a CUDA runtime call failed (message in wp_last_error) */
    WP_ERR_NONFINITE = 5, /* model contains a non-positive or non-finite value */
    WP_ERR_TIMEOUT = 6    /* a bounded device wait gave up (kernel error flag set) */
} wp_status;

enum { WP_PHYS_ISO = 0, WP_PHYS_TTI = 1 };

/* Gradient variants for wp_workspace_bytes() and wp_exact_gradient(). */
enum {
    WP_MODE_PROBED = 0,          /* forward + adjoint with probing (Eq. 3)             */
    WP_MODE_EXACT_FULL = 1,      /* full forward history kept in the workspace (Eq. 2)  */
    WP_MODE_EXACT_CHECKPOINT = 2 /* checkpoints + recomputation (Griewank/Symes, Sec. 1) */
};

typedef void *wp_stream; /* a cudaStream_t */

/* Opaque model handle (library-owned, host memory only). */
typedef struct wp_model_s wp_model_t;

/* Model description.  Device arrays are borrowed: they must outlive the handle and must
 * not change while calls using the handle are in flight. */
typedef struct {
    int ndim;          /* 2 or 3                                                   */
    int nx, ny, nz;    /* interior points per axis (ny ignored in 2-D)             */
    int nbl;           /* absorbing cells added on every side, >= 4                */
    int space_order;   /* must be 8                                                */
    int physics;       /* WP_PHYS_ISO or WP_PHYS_TTI (pseudo-acoustic, two fields) */
    double dx, dy, dz; /* grid spacing, metres                                     */
    double dt;         /* time step, seconds                                       */
    int nt;            /* number of time steps                                     */
    double damp_v;     /* velocity (m/s) scaling the absorbing layer; <= 0: the
                          maximum velocity of m                                    */
    const float *m;    /* device, N values: squared slowness (s^2/m^2), padded     */
    const float *eps, *delta, *theta, *phi; /* device, N values (user layout); TTI only:
                          Thomsen epsilon and delta, tilt theta and azimuth phi (radians;
                          phi may be NULL in 2-D).  TTI system (Sec. 3 "2007 BP TTI"):
                          m p_tt = (1+2eps) H0 p + sqrt(1+2delta) Hz q + src,
                          m q_tt = sqrt(1+2delta) H0 p + Hz q + src, Hz = -Dr^T Dr along the
                          tilted axis, H0 = L - Hz; receivers record p; the gradient and the
                          probed projections cover both fields (outputs per shot hold the
                          p part then the q part: P_u and P_v are nshots*2*r*N).      */
} wp_model_desc;

/* Acquisition of a batch of shots.  Positions are host arrays in metres measured from
 * the first interior grid point, (x, y, z) triples (y ignored in 2-D).  Each position
 * must lie strictly inside the padded grid; off-grid points use bilinear (2-D) or
 * trilinear (3-D) weights for injection and interpolation. */
typedef struct {
    int nshots;
    int nsrc;               /* sources per shot (all fire the same wavelet) */
    int nrec;               /* receivers per shot                           */
    const double *src_xyz;  /* host, nshots*nsrc*3 */
    const double *rec_xyz;  /* host, nshots*nrec*3 */
} wp_geom;

/*
 * wp_model — validate a model and create its handle (Sec. 2.2 physics).
 * Checks sizes, that every m value is finite and positive, and the stability limit
 * dt^2 v_max^2 * 6.5016 * sum_axes 1/h^2 <= 4 (8th-order leapfrog; for TTI v_max is
 * scaled by sqrt(1 + 2 max eps)); for TTI also that delta <= eps everywhere (the
 * two-field system has a growing mode where delta > eps: WP_ERR_UNSTABLE).  The checks run
 * as reductions on a stream of the library that does not wait for other streams, and the
 * call waits for that stream only: m and the Thomsen fields must already be complete on the
 * device (synchronise the stream or event that wrote them).  On success *out receives the
 * handle.
 * Returns WP_ERR_INVALID, WP_ERR_NONFINITE, WP_ERR_UNSTABLE or WP_ERR_CUDA on failure.
 */
wp_status wp_model(const wp_model_desc *desc, wp_model_t **out);

/* wp_model_free — release a handle (NULL is ignored). */
void wp_model_free(wp_model_t *model);

/* Padded point count N of a model, or -1 for NULL. */
long long wp_model_npoints(const wp_model_t *model);

/* Maximum velocity of the model (m/s), as found by wp_model(). */
double wp_model_vmax(const wp_model_t *model);

/*
 * Layout of the probed projections P_u and P_v that wp_probe_forward writes,
 * wp_adjoint_image reads and writes, and wp_offset_image reads (Eq. 3, Eq. 4), chosen per
 * model handle (the default is WP_PROBES_DENSE):
 *   WP_PROBES_DENSE    row (shot, probe) holds the model's N points, x fastest; rows are N
 *                      floats apart.  The library accumulates in the aligned layout and
 *                      copies into this one once per call (one read and one write of P).
 *   WP_PROBES_ALIGNED  rows are row_floats floats apart (N_aligned rounded up to 128, so
 *                      every row starts on a 512-byte boundary) and point (x, y, z) of a
 *                      row sits at ((z * NY + y) * x_pitch + x), where x_pitch is the padded
 *                      NX rounded up to 4 and NY the padded y count (y = 0 in 2-D).  The
 *                      contraction writes these rows directly (no copy), and
 *                      wp_offset_image loads them as 16-byte vectors.  Entries at
 *                      x >= NX and past the last point of a row hold unspecified values.
 *                      Buffers hold nshots * r * row_floats floats (TTI: 2 * nshots * r
 *                      rows) and must be 16-byte aligned.
 * wp_set_probe_layout returns WP_ERR_INVALID for a NULL model or an unknown layout; it
 * must not be called while calls using the handle are in flight.  wp_probe_layout reports
 * the layout and, for it, the floats between rows and the x pitch (any output may be NULL;
 * dense: N and NX).
 */
enum { WP_PROBES_DENSE = 0, WP_PROBES_ALIGNED = 1 };
wp_status wp_set_probe_layout(wp_model_t *model, int layout);
wp_status wp_probe_layout(const wp_model_t *model, int *layout, long long *row_floats, int *x_pitch);

/*
 * wp_workspace_bytes — device scratch needed by one call of the given mode for this
 * model, acquisition, probe count r and probe block Tb (buffered time steps per
 * tensor-core contraction; a multiple of 16).  For WP_MODE_EXACT_CHECKPOINT, Tb is the
 * checkpoint interval in steps.  This is also the admission quantity: the memory the
 * method needs per batch of shots.  Returns 0 on invalid arguments.
 */
size_t wp_workspace_bytes(const wp_model_t *model, const wp_geom *geom, int r, int Tb, int mode);

/*
 * wp_probe_forward — forward propagation with on-the-fly probing (Eq. 3, Eq. 1).
 *   wavelet  device, nt values: the source time function injected at every source
 *   Q        device, nshots*nt*r values: probing matrix of shot s, row t (time), column i;
 *            Rademacher +-1 or any orthonormal basis (row-major, nt x r per shot)
 *   r        number of probes, 0..512 (0: plain modelling, P_u unused); the contraction
 *            reads each block of the wavefield once for all r probes
 *   Tb       time steps buffered between tensor-core contractions, multiple of 16
 *   P_u      device out, nshots*r rows in the model's probe layout (wp_set_probe_layout):
 *            P_u[s][i][x] = sum_t Q[s][t][i] u_tt[s][t][x]
 *   d_syn    device out, nshots*nt*nrec (row t = R u^{t+1}) or NULL
 *   ws       device workspace of at least wp_workspace_bytes(.., WP_MODE_PROBED) bytes
 */
wp_status wp_probe_forward(wp_model_t *model, const wp_geom *geom, const float *wavelet,
                           const float *Q, int r, int Tb, float *P_u, float *d_syn,
                           void *ws, size_t ws_bytes, wp_stream stream);

/*
 * wp_adjoint_image — adjoint propagation with on-the-fly probing and the randomized
 * imaging condition (Eq. 3), summed over the shots of the batch.
 *   residual  device, nshots*nt*nrec: d_syn - d_obs (row t is injected at adjoint step t)
 *   Q, r, Tb  as in wp_probe_forward (the same Q must be used, Eq. 3)
 *   scale     estimator normalisation: 1/r for Rademacher probes, 1 for orthonormal Q
 *   P_u       device, from wp_probe_forward (the model's probe layout)
 *   g         device out, N: sum_s scale * sum_i P_u[s][i] * P_v[s][i]
 *   P_v       device out, nshots*r rows in the model's probe layout, or NULL (then kept in
 *             the workspace)
 */
wp_status wp_adjoint_image(wp_model_t *model, const wp_geom *geom, const float *residual,
                           const float *Q, int r, int Tb, float scale, const float *P_u,
                           float *g, float *P_v, void *ws, size_t ws_bytes, wp_stream stream);

/*
 * wp_exact_gradient — the exact adjoint-state gradient (Eq. 2) summed over the batch,
 * the baseline the probed method is measured against.
 *   mode     WP_MODE_EXACT_FULL: the whole forward history stays in the workspace;
 *            WP_MODE_EXACT_CHECKPOINT: states every `ncheck` steps are stored and each
 *            segment is recomputed once during the adjoint sweep (Sec. 1, optimal
 *            checkpointing, two levels)
 *   ncheck   checkpoint interval in steps (checkpoint mode; must equal the Tb given to
 *            wp_workspace_bytes)
 *   d_obs    device, nshots*nt*nrec observed data
 *   g        device out, N
 *   misfit   device out, one double: J = 1/2 sum |d_syn - d_obs|^2, or NULL
 *   d_syn    device out, nshots*nt*nrec, or NULL
 */
wp_status wp_exact_gradient(wp_model_t *model, const wp_geom *geom, const float *wavelet,
                            const float *d_obs, float *g, double *misfit, float *d_syn,
                            int mode, int ncheck, void *ws, size_t ws_bytes, wp_stream stream);

/*
 * wp_offset_image — the subsurface-offset image volume (Eq. 4) from probed projections,
 * summed over the shots of the batch:
 *   out[h + nh][p] = scale * sum_s sum_i P_u[s][i][p + h] * P_v[s][i][p - h],  h = -nh..nh,
 * where p + h moves h points along x (the fastest axis of the padded grid) and terms whose
 * shifted point leaves the x-row are zero.  Offset 0 equals the image of wp_adjoint_image.
 *   P_u, P_v  device, nshots*r rows in the model's probe layout, as written by
 *             wp_probe_forward and wp_adjoint_image (P_v must have been requested there);
 *             16-byte aligned in WP_PROBES_ALIGNED
 *   scale     estimator normalisation as in wp_adjoint_image
 *   r         1..512
 *   nh        0 <= nh <= 64 offsets on each side (the paper's gathers: 40 at 12.5 m)
 *   out       device out, (2*nh + 1)*N floats (dense, x fastest), overwritten
 * Per (z, y) row the volume is a band of the Gram matrix P_u^T P_v over k = (shot, probe),
 * computed on the tensor cores (bf16 hi/lo split of both operands, FP32 accumulation:
 * about 3.5e-6 relative error on random projections).  WP_ERR_INVALID for bad arguments;
 * asynchronous on `stream`; wp_offset_status() reports a device wait that gave up.
 */
wp_status wp_offset_image(const wp_model_t *model, const float *P_u, const float *P_v, int r,
                          int nshots, float scale, int nh, float *out, wp_stream stream);

/* wp_offset_status — polls `stream` from the host for at most timeout_s seconds, then
 * reads the error flag of the offset-volume kernel (WP_ERR_TIMEOUT if either fails). */
wp_status wp_offset_status(wp_stream stream, double timeout_s);

/*
 * wp_residual — res = d_syn - d_obs (n values) and, if misfit != NULL, the device double
 * J = 1/2 sum res^2 (deterministic two-pass reduction).  `ws` needs
 * wp_residual_workspace_bytes(n) bytes (may be NULL when misfit is NULL).
 */
wp_status wp_residual(const float *d_syn, const float *d_obs, float *res, long long n,
                      double *misfit, void *ws, size_t ws_bytes, wp_stream stream);
size_t wp_residual_workspace_bytes(long long n);

/*
 * wp_probe_accumulate — the tensor-core probe contraction alone (Eq. 3 block update):
 * for each shot s and point x,
 *   P[s][i][x] += scale * sum_{t<cnt} A[s][t][x] * Q[s][t0 + t][i]
 * where A[s] is a cnt x N block (row t contiguous over x, shot stride cnt*N) and Q is as
 * in wp_probe_forward, 1 <= r <= 512.  Both operands are split into bfloat16 hi/lo pairs
 * and multiplied with FP32 accumulation (tcgen05).  `ws` needs
 * wp_probe_accumulate_workspace_bytes().
 */
wp_status wp_probe_accumulate(const float *A, int cnt, long long npoints, int nshots,
                              const float *Q, int nt, int t0, int r, float scale, float *P,
                              void *ws, size_t ws_bytes, wp_stream stream);
size_t wp_probe_accumulate_workspace_bytes(int nshots, int nt, int r);

/*
 * wp_probe_accumulate_static — the same contraction as wp_probe_accumulate for callers
 * that cannot provide any device scratch memory: code that only holds device pointers to
 * its own inputs and outputs, for instance a plug-in inside an application whose
 * framework owns the whole GPU through its own allocator, or a service whose memory
 * budget is fixed.  The paper has no counterpart; this is a deployment variant.
 *   - Scratch (the bf16 hi/lo copy of Q and an error flag) lives in a 16 MiB device
 *     array inside libwp.so, reserved on every GPU that loads the library until the
 *     process exits.  Requires 256 + 2 * nshots * r_pad * nt_pad * 2 bytes <= 16 MiB with
 *     r_pad = max(16, r rounded up to 16) and nt_pad = nt rounded up to 64, plus 64;
 *     larger requests return WP_ERR_OOM.  No device memory is allocated.
 *   - The first call on a device looks up the array's device address for that device
 *     (cudaGetSymbolAddress); make that first call before any stream capture.  The
 *     address is kept with the id of the context it was found in, so the first call after
 *     a cudaDeviceReset looks it up again.
 *   - Every call on a device shares the one array: calls whose work overlaps on the GPU
 *     (other streams, other threads) race and must be serialised by the caller.
 *   - A device wait that gives up sets an error flag inside the array: read it with
 *     wp_static_status() after the call.
 * Arguments as in wp_probe_accumulate.
 */
wp_status wp_probe_accumulate_static(const float *A, int cnt, long long npoints, int nshots,
                                     const float *Q, int nt, int t0, int r, float scale,
                                     float *P, wp_stream stream);

/*
 * wp_range_finder — range-finder probing vectors (Sec. 2.1: [Q, ~] = qr(A Z), the
 * randomized range finder of the traced matrix), for a batch of shots:
 *   Q[s] = orth((D_s D_s^T)^power Z[s])
 * with orth the thin QR's Q whose R has a positive diagonal.  The paper leaves A open;
 * A = D D^T covers this library's two readings: D the shot's nt x nrec data (ncols =
 * nrec) or the nt x nt causal convolution matrix of the source wavelet.  Use the result
 * as the probing matrix of wp_probe_forward / wp_adjoint_image with scale 1.
 *   D        device, nt x ncols row-major per shot (shot stride nt*ncols), or one matrix
 *            for all shots when d_shared != 0
 *   Z        device, nshots*nt*r: the sketch's random matrix (e.g. Rademacher), row t
 *   power    1..8 applications of D D^T (power iteration; Q is re-orthonormalised after
 *            each, which leaves the final Q unchanged in exact arithmetic)
 *   r        1 <= r <= min(256, nt)
 *   Q        device out, nshots*nt*r, row-major (t, i) like the probe input of the calls
 *            above
 *   ws       device workspace of wp_range_finder_workspace_bytes() bytes; its first bytes
 *            hold the error flag that wp_stream_status(ws, ...) reads (a rank-deficient
 *            sketch raises it and gets zero columns)
 * Both products of a power step run on the tensor-core contraction (bf16 hi/lo split,
 * FP32 accumulation); the QR is classical Gram-Schmidt with one reorthogonalisation in
 * FP64, one CTA per shot.  WP_ERR_INVALID / WP_ERR_OOM on bad arguments; asynchronous.
 */
size_t wp_range_finder_workspace_bytes(int nt, int ncols, int nshots, int d_shared, int r);
wp_status wp_range_finder(const float *D, int nt, int ncols, int nshots, int d_shared, int power,
                          const float *Z, int r, float *Q, void *ws, size_t ws_bytes,
                          wp_stream stream);

/*
 * wp_static_status — status of the last wp_probe_accumulate_static call on the current
 * device (the paper has no counterpart): polls `stream` from the host for at most
 * timeout_s seconds, then reads the error flag kept in the static array (a device-to-host
 * copy of 4 bytes, no allocation).  WP_ERR_TIMEOUT if the deadline passed or a bounded
 * device wait gave up.
 */
wp_status wp_static_status(wp_stream stream, double timeout_s);

/*
 * wp_stream_status — wait for `stream` by polling it from the host (never spinning on the
 * device) for at most timeout_s seconds, then read the device error flag that every
 * workspace keeps in its first bytes (`ws` may be NULL to skip that check).  Returns
 * WP_ERR_TIMEOUT if the deadline passed or a bounded device wait gave up.
 */
wp_status wp_stream_status(const void *ws, wp_stream stream, double timeout_s);

/*
 * wp_check_bounded_wait — diagnostic of the failure path: clears the error flag in the first
 * bytes of `ws` (at least 256 bytes, 16-byte aligned device memory) and launches on `stream`
 * one thread that waits on a shared-memory mbarrier no copy or thread ever completes.  The
 * wait gives up after about 2^31 clock cycles (about one second), sets the flag and returns,
 * so the following wp_stream_status(ws, ...) reports WP_ERR_TIMEOUT and the context stays
 * usable.  WP_ERR_INVALID for a missing or short workspace; asynchronous on `stream`.
 */
wp_status wp_check_bounded_wait(void *ws, size_t ws_bytes, wp_stream stream);

/*
 * Optional kernel timing for measurement: wp_profile_enable(1, capacity) makes the library
 * record a CUDA event pair on the launching stream around each of the next `capacity`
 * launches of every kernel class (0 = one-step stencil launch, 1 = probe contraction,
 * 2 = other, 3 = two-step stencil launch, 4 = two-step launch of the exact adjoint with the
 * imaging condition; -1 from wp_profile_read for an unknown class);
 * wp_profile_enable(0, 0) stops recording.  After the caller has synchronised,
 * wp_profile_read(class, &total_ms, &count) returns the summed device time of the
 * recorded launches.  Not thread-safe; intended for benchmarks.
 */
void wp_profile_enable(int on, int capacity);
int wp_profile_read(int cls, double *total_ms, long long *count);

/* Thread-local description of the last failure ("" if none). */
const char *wp_last_error(void);

/* Number of kernels this host process has launched through the library. */
long long wp_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* WP_H */
