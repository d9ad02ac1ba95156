/*
 * FP64 CPU oracle for the probed (randomized-trace) adjoint-state gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline may load this library.  It shares no code, header, table or helper with the
 * CUDA path in paper_2201_06914_gb300/csrc; both sides receive the same seeded inputs.
 *
 * What it computes, in the order and notation of the paper (Louboutin & Herrmann,
 * "Enabling wave-based inversion on GPUs with randomized trace estimation"):
 *
 *   - Sec. 2.2: the isotropic acoustic wave equation, which the paper names but does not
 *     write out, read as  m (u_tt + sigma u_t) - Laplacian(u) = q,  m = 1/v^2, sigma a
 *     fixed absorbing-layer damping rate (1/s) that is zero inside the model.  Time is a
 *     2nd-order centred difference, space the 8th-order textbook central difference.
 *     Zero Dirichlet values lie beyond the padded grid.
 *   - Eq. 2: the exact gradient  dm = sum_t u_tt[t] v[t]  (the discrete dJ/dm of
 *     J = 1/2 sum_t |R u[t] - d_obs[t]|^2), with u_tt the m-derivative of the discrete
 *     operator at step t (in the model interior exactly the centred second difference
 *     of u divided by dt^2) and v the adjoint wavefield scaled so that Eq. 2 carries no
 *     extra factor.
 *   - Eq. 3: projections  Pu = Q^T u_tt,  Pv = Q^T v  accumulated one time step at a time,
 *     and the estimate  dm[x] ~= s * sum_i Pu[i,x] Pv[i,x]  (s = 1/r for Rademacher Q,
 *     s = 1 for orthonormal Q).
 *
 * Discrete scheme (one shot), n = 0 .. nt-1, u^0 = u^-1 = 0:
 *   m[(u^{n+1} - 2u^n + u^{n-1})/dt^2 + sigma (u^{n+1} - u^{n-1})/(2dt)] = L u^n + q^n
 *   u_tt^n = (u^{n+1} - 2u^n + u^{n-1})/dt^2 + sigma (u^{n+1} - u^{n-1})/(2dt)
 *   d[n]   = R u^{n+1}                                   (bilinear/trilinear interpolation)
 *   q^n    = sum_sources w * wavelet[n] (+ an optional volume source)
 * Adjoint, j = nt-1 .. 0, v^{nt} = v^{nt+1} = 0:
 *   m[(v^j - 2v^{j+1} + v^{j+2})/dt^2 + sigma (v^j - v^{j+2})/(2dt)] = L v^{j+1} - R^T res[j]
 *   gradient  g = sum_j u_tt^j * v^j,   Pv[i] = sum_j Q[j,i] v^j
 * With this scaling g equals dJ/dm exactly (checked by the Born dot test and the Taylor
 * test in tests/), so the sign and factor readings of Eq. 2 are pinned there.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int ndim, nx, ny, nz, nbl, nt;
    double dx, dy, dz, dt;
    double damp_v; /* velocity (m/s) that sets the absorbing-layer strength */
} orc_grid;

/* 8th-order central second-derivative weights (Fornberg 1988): offsets 0..4. */
static const double FD2[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

static void dims(const orc_grid *g, long *NX, long *NY, long *NZ)
{
    *NX = g->nx + 2L * g->nbl;
    *NY = (g->ndim == 3) ? g->ny + 2L * g->nbl : 1;
    *NZ = g->nz + 2L * g->nbl;
}

long orc_npoints(const orc_grid *g)
{
    long NX, NY, NZ;
    dims(g, &NX, &NY, &NZ);
    return NX * NY * NZ;
}

/* Damping rate on one axis: sigma0 (d/nbl)^2 with d the depth (cells) into the layer and
 * sigma0 = 3 v ln(1000) / (2 nbl h). */
static double damp_axis(long i, long n, long nbl, double h, double v)
{
    double d = 0.0;
    if (i < nbl) d = (double)(nbl - i);
    else if (i >= nbl + n) d = (double)(i - (nbl + n - 1));
    double s0 = 3.0 * v * log(1000.0) / (2.0 * nbl * h);
    return s0 * (d / nbl) * (d / nbl);
}

void orc_sponge(const orc_grid *g, double *sigma)
{
    long NX, NY, NZ;
    dims(g, &NX, &NY, &NZ);
    for (long z = 0; z < NZ; z++)
        for (long y = 0; y < NY; y++)
            for (long x = 0; x < NX; x++) {
                double s = damp_axis(x, g->nx, g->nbl, g->dx, g->damp_v) +
                           damp_axis(z, g->nz, g->nbl, g->dz, g->damp_v);
                if (g->ndim == 3) s += damp_axis(y, g->ny, g->nbl, g->dy, g->damp_v);
                sigma[(z * NY + y) * NX + x] = s;
            }
}

/* Corner indices and bilinear (2-D) / trilinear (3-D) weights of a point given in metres
 * from the first interior point.  Returns the corner count, or -1 when the point is not
 * strictly inside the padded grid. */
int orc_weights(const orc_grid *g, const double *xyz, long *idx, double *w)
{
    long NX, NY, NZ;
    dims(g, &NX, &NY, &NZ);
    double gx = g->nbl + xyz[0] / g->dx, gz = g->nbl + xyz[2] / g->dz;
    double gy = (g->ndim == 3) ? g->nbl + xyz[1] / g->dy : 0.0;
    if (gx < 0 || gx >= NX - 1 || gz < 0 || gz >= NZ - 1) return -1;
    if (g->ndim == 3 && (gy < 0 || gy >= NY - 1)) return -1;
    long ix = (long)floor(gx), iy = (long)floor(gy), iz = (long)floor(gz);
    double fx = gx - ix, fy = gy - iy, fz = gz - iz;
    int nc = 0;
    int ny_c = (g->ndim == 3) ? 2 : 1;
    for (int cz = 0; cz < 2; cz++)
        for (int cy = 0; cy < ny_c; cy++)
            for (int cx = 0; cx < 2; cx++) {
                double wx = cx ? fx : 1.0 - fx, wz = cz ? fz : 1.0 - fz;
                double wy = (g->ndim == 3) ? (cy ? fy : 1.0 - fy) : 1.0;
                idx[nc] = ((iz + cz) * NY + (iy + cy)) * NX + (ix + cx);
                w[nc] = wx * wy * wz;
                nc++;
            }
    return nc;
}

/* out = L u, the 8th-order Laplacian with zero values beyond the padded grid. */
static void laplacian(const orc_grid *g, const double *u, double *out)
{
    long NX, NY, NZ;
    dims(g, &NX, &NY, &NZ);
    const double ihx = 1.0 / (g->dx * g->dx), ihz = 1.0 / (g->dz * g->dz);
    const double ihy = (g->ndim == 3) ? 1.0 / (g->dy * g->dy) : 0.0;
#pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < NZ; z++)
        for (long y = 0; y < NY; y++)
            for (long x = 0; x < NX; x++) {
                long p = (z * NY + y) * NX + x;
                double sx = FD2[0] * u[p], sz = FD2[0] * u[p], sy = FD2[0] * u[p];
                for (int k = 1; k <= 4; k++) {
                    if (x - k >= 0) sx += FD2[k] * u[p - k];
                    if (x + k < NX) sx += FD2[k] * u[p + k];
                    if (z - k >= 0) sz += FD2[k] * u[p - k * NX * NY];
                    if (z + k < NZ) sz += FD2[k] * u[p + k * NX * NY];
                    if (g->ndim == 3) {
                        if (y - k >= 0) sy += FD2[k] * u[p - k * NX];
                        if (y + k < NY) sy += FD2[k] * u[p + k * NX];
                    }
                }
                out[p] = sx * ihx + sz * ihz + (g->ndim == 3 ? sy * ihy : 0.0);
            }
}

/* Exported for the tests: out = L u on the padded grid. */
void orc_apply_laplacian(const orc_grid *g, const double *u, double *out) { laplacian(g, u, out); }

/* One leapfrog step of  m[(w_new - 2w + w_old)/dt^2 + sigma (w_new - w_old)/(2dt)] = L w + q,
 * solved for w_new.  `lq` holds L w + q on entry. */
static void leapfrog(long N, double dt, const double *m, const double *sigma, const double *lq,
                     const double *w, const double *w_old, double *w_new)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; p++) {
        double a = m[p] / (dt * dt), b = m[p] * sigma[p] / (2.0 * dt);
        /* (a + b) w_new = lq + 2a w - (a - b) w_old */
        w_new[p] = (lq[p] + 2.0 * a * w[p] - (a - b) * w_old[p]) / (a + b);
    }
}

/*
 * Forward propagation of one shot (Sec. 2.2) with on-the-fly probing (Eq. 3).
 *   m        padded squared slowness, N values
 *   src_xyz  nsrc points (metres), each injecting wavelet[n] at step n
 *   vol_src  optional nt*N volume source added to q^n (NULL for none)
 *   d        out nt*nrec, row n = R u^{n+1}            (NULL to skip)
 *   Q, r     probing matrix nt*r (row n) and its width  (r = 0 to skip)
 *   Pu       out r*N: Pu[i] = sum_n Q[n,i] u_tt^n        (overwritten)
 *   udd      out nt*N: u_tt^n                           (NULL to skip)
 *   uhist    out (nt+1)*N: u^0 .. u^nt                  (NULL to skip)
 * Returns 0, or -1 when a source or receiver lies outside the grid.
 */
int orc_forward(const orc_grid *g, const double *m, int nsrc, const double *src_xyz,
                const double *wavelet, const double *vol_src, int nrec, const double *rec_xyz,
                double *d, int r, const double *Q, double *Pu, double *udd, double *uhist)
{
    const long N = orc_npoints(g);
    const int nt = g->nt;
    const double dt = g->dt;
    long (*sidx)[8] = calloc((size_t)(nsrc > 0 ? nsrc : 1), sizeof(*sidx));
    double (*sw)[8] = calloc((size_t)(nsrc > 0 ? nsrc : 1), sizeof(*sw));
    long (*ridx)[8] = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(*ridx));
    double (*rw)[8] = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(*rw));
    int *snc = calloc((size_t)(nsrc > 0 ? nsrc : 1), sizeof(int));
    int *rnc = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(int));
    double *sigma = malloc(N * sizeof(double));
    double *u_old = calloc(N, sizeof(double)), *u = calloc(N, sizeof(double));
    double *u_new = calloc(N, sizeof(double)), *lq = malloc(N * sizeof(double));
    int rc = 0;
    for (int s = 0; s < nsrc; s++)
        if ((snc[s] = orc_weights(g, src_xyz + 3 * s, sidx[s], sw[s])) < 0) rc = -1;
    for (int j = 0; j < nrec; j++)
        if ((rnc[j] = orc_weights(g, rec_xyz + 3 * j, ridx[j], rw[j])) < 0) rc = -1;
    if (rc) goto done;
    orc_sponge(g, sigma);
    if (r > 0 && Pu) memset(Pu, 0, (size_t)r * N * sizeof(double));
    if (uhist) memset(uhist, 0, N * sizeof(double));
    for (int n = 0; n < nt; n++) {
        laplacian(g, u, lq);
        if (vol_src)
            for (long p = 0; p < N; p++) lq[p] += vol_src[(long)n * N + p];
        for (int s = 0; s < nsrc; s++)
            for (int c = 0; c < snc[s]; c++) lq[sidx[s][c]] += sw[s][c] * wavelet[n];
        leapfrog(N, dt, m, sigma, lq, u, u_old, u_new);
        /* u_tt^n: the m-derivative of the discrete operator (Eq. 2's second derivative) */
        double *a = lq; /* reuse */
#pragma omp parallel for schedule(static)
        for (long p = 0; p < N; p++)
            a[p] = (u_new[p] - 2.0 * u[p] + u_old[p]) / (dt * dt) +
                   sigma[p] * (u_new[p] - u_old[p]) / (2.0 * dt);
        if (udd) memcpy(udd + (long)n * N, a, N * sizeof(double));
        if (r > 0 && Pu) {
#pragma omp parallel for schedule(static)
            for (long p = 0; p < N; p++)
                for (int i = 0; i < r; i++) Pu[(long)i * N + p] += Q[(long)n * r + i] * a[p];
        }
        if (d)
            for (int j = 0; j < nrec; j++) {
                double acc = 0.0;
                for (int c = 0; c < rnc[j]; c++) acc += rw[j][c] * u_new[ridx[j][c]];
                d[(long)n * nrec + j] = acc;
            }
        if (uhist) memcpy(uhist + (long)(n + 1) * N, u_new, N * sizeof(double));
        double *t = u_old;
        u_old = u;
        u = u_new;
        u_new = t;
    }
done:
    free(sidx); free(sw); free(ridx); free(rw); free(snc); free(rnc);
    free(sigma); free(u_old); free(u); free(u_new); free(lq);
    return rc;
}

/*
 * Adjoint propagation of one shot with the residual injected at the receivers.
 *   res     nt*nrec, row j is injected at adjoint step j (pairs with d row j)
 *   Q, r    probing matrix; Pv out r*N, Pv[i] = sum_j Q[j,i] v^j  (r = 0 to skip)
 *   udd     nt*N forward u_tt history (NULL to skip the exact gradient)
 *   grad    out N: sum_j u_tt^j v^j  (overwritten; needs udd)
 *   vhist   out nt*N: v^j             (NULL to skip)
 *   pt_xyz, npt, vpt  optional sampling of v at points: vpt[j*npt + k] = sum_c w v^j
 */
int orc_adjoint(const orc_grid *g, const double *m, int nrec, const double *rec_xyz,
                const double *res, int r, const double *Q, double *Pv, const double *udd,
                double *grad, double *vhist, int npt, const double *pt_xyz, double *vpt)
{
    const long N = orc_npoints(g);
    const int nt = g->nt;
    const double dt = g->dt;
    long (*ridx)[8] = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(*ridx));
    double (*rw)[8] = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(*rw));
    int *rnc = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(int));
    long (*pidx)[8] = calloc((size_t)(npt > 0 ? npt : 1), sizeof(*pidx));
    double (*pw)[8] = calloc((size_t)(npt > 0 ? npt : 1), sizeof(*pw));
    int *pnc = calloc((size_t)(npt > 0 ? npt : 1), sizeof(int));
    double *sigma = malloc(N * sizeof(double));
    double *v2 = calloc(N, sizeof(double)), *v1 = calloc(N, sizeof(double));
    double *v0 = calloc(N, sizeof(double)), *lq = malloc(N * sizeof(double));
    int rc = 0;
    for (int j = 0; j < nrec; j++)
        if ((rnc[j] = orc_weights(g, rec_xyz + 3 * j, ridx[j], rw[j])) < 0) rc = -1;
    for (int k = 0; k < npt; k++)
        if ((pnc[k] = orc_weights(g, pt_xyz + 3 * k, pidx[k], pw[k])) < 0) rc = -1;
    if (rc) goto done;
    orc_sponge(g, sigma);
    if (r > 0 && Pv) memset(Pv, 0, (size_t)r * N * sizeof(double));
    if (grad) memset(grad, 0, N * sizeof(double));
    for (int j = nt - 1; j >= 0; j--) {
        laplacian(g, v1, lq);
        for (int k = 0; k < nrec; k++)
            for (int c = 0; c < rnc[k]; c++) lq[ridx[k][c]] -= rw[k][c] * res[(long)j * nrec + k];
        leapfrog(N, dt, m, sigma, lq, v1, v2, v0);
        if (vhist) memcpy(vhist + (long)j * N, v0, N * sizeof(double));
        if (r > 0 && Pv) {
#pragma omp parallel for schedule(static)
            for (long p = 0; p < N; p++)
                for (int i = 0; i < r; i++) Pv[(long)i * N + p] += Q[(long)j * r + i] * v0[p];
        }
        if (grad && udd) {
#pragma omp parallel for schedule(static)
            for (long p = 0; p < N; p++) grad[p] += udd[(long)j * N + p] * v0[p];
        }
        for (int k = 0; k < npt; k++) {
            double acc = 0.0;
            for (int c = 0; c < pnc[k]; c++) acc += pw[k][c] * v0[pidx[k][c]];
            vpt[(long)j * npt + k] = acc;
        }
        double *t = v2;
        v2 = v1;
        v1 = v0;
        v0 = t;
    }
done:
    free(ridx); free(rw); free(rnc); free(pidx); free(pw); free(pnc);
    free(sigma); free(v2); free(v1); free(v0); free(lq);
    return rc;
}

/* Eq. 3: out[x] = scale * sum_i Pu[i,x] Pv[i,x]. */
void orc_probed_image(long N, int r, const double *Pu, const double *Pv, double scale, double *out)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; p++) {
        double acc = 0.0;
        for (int i = 0; i < r; i++) acc += Pu[(long)i * N + p] * Pv[(long)i * N + p];
        out[p] = scale * acc;
    }
}


/* ======================================================================================
 * Pseudo-acoustic TTI (the paper's second physics, Sec. 3 "2007 BP TTI"; equations not
 * given in the paper).  Reading: the two-field system
 *   m (p_tt + sigma p_t) = (1 + 2 eps) H0 p + sqrt(1 + 2 delta) Hz q + q_src
 *   m (q_tt + sigma q_t) = sqrt(1 + 2 delta) H0 p + Hz q + q_src
 * with Hz = -Dr^T Dr, Dr = ax Dx + ay Dy + az Dz (8th-order central first derivatives,
 * ax = sin(theta) cos(phi), ay = sin(theta) sin(phi), az = cos(theta)) and H0 = L - Hz.
 * Both Hz and H0 are symmetric; the block operator is not, so the adjoint applies its
 * transpose: [H0 (E a + S b); Hz (S a + b)] with E = 1 + 2 eps, S = sqrt(1 + 2 delta).
 * The source fires in both fields; the receivers record p; the gradient sums both fields:
 * g = sum_t (p_tt v_p + q_tt v_q).
 * ====================================================================================== */

/* 8th-order central first-derivative weights for offsets 1..4 (antisymmetric). */
static const double FD1[5] = {0.0, 4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};

/* out = d/d(axis) u, axis 0 = x, 1 = y, 2 = z; zero values beyond the grid. */
static void deriv1(const orc_grid *g, const double *u, double *out, int axis)
{
    long NX, NY, NZ;
    dims(g, &NX, &NY, &NZ);
    const double h = axis == 0 ? g->dx : axis == 1 ? g->dy : g->dz;
    const long st = axis == 0 ? 1 : axis == 1 ? NX : NX * NY;
#pragma omp parallel for collapse(2) schedule(static)
    for (long z = 0; z < NZ; z++)
        for (long y = 0; y < NY; y++)
            for (long x = 0; x < NX; x++) {
                const long p = (z * NY + y) * NX + x;
                const long i = axis == 0 ? x : axis == 1 ? y : z;
                const long n = axis == 0 ? NX : axis == 1 ? NY : NZ;
                double acc = 0.0;
                for (int k = 1; k <= 4; k++) {
                    if (i + k < n) acc += FD1[k] * u[p + k * st];
                    if (i - k >= 0) acc -= FD1[k] * u[p - k * st];
                }
                out[p] = acc / h;
            }
}

typedef struct {
    long N;
    double *t, *d, *w;   /* scratch, N each */
    const double *ax, *ay, *az;
    int ndim;
} tti_work;

/* out = Hz w = -Dr^T Dr w = sum_i D_i (a_i Dr w)  (D_i^T = -D_i). */
static void apply_hz(const orc_grid *g, tti_work *T, const double *w, double *out)
{
    const long N = T->N;
    deriv1(g, w, T->d, 0);
    for (long p = 0; p < N; p++) T->t[p] = T->ax[p] * T->d[p];
    if (T->ndim == 3) {
        deriv1(g, w, T->d, 1);
        for (long p = 0; p < N; p++) T->t[p] += T->ay[p] * T->d[p];
    }
    deriv1(g, w, T->d, 2);
    for (long p = 0; p < N; p++) T->t[p] += T->az[p] * T->d[p];
    for (long p = 0; p < N; p++) T->w[p] = T->ax[p] * T->t[p];
    deriv1(g, T->w, out, 0);
    if (T->ndim == 3) {
        for (long p = 0; p < N; p++) T->w[p] = T->ay[p] * T->t[p];
        deriv1(g, T->w, T->d, 1);
        for (long p = 0; p < N; p++) out[p] += T->d[p];
    }
    for (long p = 0; p < N; p++) T->w[p] = T->az[p] * T->t[p];
    deriv1(g, T->w, T->d, 2);
    for (long p = 0; p < N; p++) out[p] += T->d[p];
}

/* Exported for the tests: out = Hz w for the given angles. */
void orc_apply_hz(const orc_grid *g, const double *theta, const double *phi, const double *w,
                  double *out)
{
    const long N = orc_npoints(g);
    double *ax = malloc(N * sizeof(double)), *ay = malloc(N * sizeof(double));
    double *az = malloc(N * sizeof(double));
    for (long p = 0; p < N; p++) {
        const double ph = phi ? phi[p] : 0.0;
        ax[p] = sin(theta[p]) * cos(ph);
        ay[p] = sin(theta[p]) * sin(ph);
        az[p] = cos(theta[p]);
    }
    tti_work T = {N, malloc(N * sizeof(double)), malloc(N * sizeof(double)),
                  malloc(N * sizeof(double)), ax, ay, az, g->ndim};
    apply_hz(g, &T, w, out);
    free(T.t); free(T.d); free(T.w); free(ax); free(ay); free(az);
}

static void tti_setup(const orc_grid *g, const double *eps, const double *delta,
                      const double *theta, const double *phi, double **E, double **S,
                      double **ax, double **ay, double **az)
{
    const long N = orc_npoints(g);
    *E = malloc(N * sizeof(double));
    *S = malloc(N * sizeof(double));
    *ax = malloc(N * sizeof(double));
    *ay = malloc(N * sizeof(double));
    *az = malloc(N * sizeof(double));
    for (long p = 0; p < N; p++) {
        (*E)[p] = 1.0 + 2.0 * eps[p];
        (*S)[p] = sqrt(1.0 + 2.0 * delta[p]);
        const double ph = (g->ndim == 3 && phi) ? phi[p] : 0.0;
        (*ax)[p] = sin(theta[p]) * cos(ph);
        (*ay)[p] = sin(theta[p]) * sin(ph);
        (*az)[p] = cos(theta[p]);
    }
}

/*
 * TTI forward of one shot.  Outputs as orc_forward, per field: Pu is 2*r*N (field p then
 * field q), udd is nt*2*N (p_tt then q_tt per step).  The volume source (Born) is 2*nt*N:
 * step n holds the p part then the q part.
 */
int orc_tti_forward(const orc_grid *g, const double *m, const double *eps, const double *delta,
                    const double *theta, const double *phi, int nsrc, const double *src_xyz,
                    const double *wavelet, const double *vol_src, int nrec, const double *rec_xyz,
                    double *d, int r, const double *Q, double *Pu, double *udd)
{
    const long N = orc_npoints(g);
    const int nt = g->nt;
    const double dt = g->dt;
    double *E, *S, *ax, *ay, *az;
    tti_setup(g, eps, delta, theta, phi, &E, &S, &ax, &ay, &az);
    tti_work T = {N, malloc(N * sizeof(double)), malloc(N * sizeof(double)),
                  malloc(N * sizeof(double)), ax, ay, az, g->ndim};
    long sidx[64][8];
    double sw[64][8];
    int snc[64];
    long (*ridx)[8] = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(*ridx));
    double (*rw)[8] = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(*rw));
    int *rnc = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(int));
    double *sigma = malloc(N * sizeof(double));
    double *p0 = calloc(N, sizeof(double)), *p1 = calloc(N, sizeof(double)), *p2 = calloc(N, sizeof(double));
    double *q0 = calloc(N, sizeof(double)), *q1 = calloc(N, sizeof(double)), *q2 = calloc(N, sizeof(double));
    double *Lp = malloc(N * sizeof(double)), *Hp = malloc(N * sizeof(double));
    double *Hq = malloc(N * sizeof(double)), *rp = malloc(N * sizeof(double));
    double *rq = malloc(N * sizeof(double));
    int rc = 0;
    if (nsrc > 64) rc = -1;
    for (int s = 0; s < nsrc && !rc; s++)
        if ((snc[s] = orc_weights(g, src_xyz + 3 * s, sidx[s], sw[s])) < 0) rc = -1;
    for (int j = 0; j < nrec && !rc; j++)
        if ((rnc[j] = orc_weights(g, rec_xyz + 3 * j, ridx[j], rw[j])) < 0) rc = -1;
    if (rc) goto done;
    orc_sponge(g, sigma);
    if (r > 0 && Pu) memset(Pu, 0, (size_t)2 * r * N * sizeof(double));
    for (int n = 0; n < nt; n++) {
        laplacian(g, p1, Lp);
        apply_hz(g, &T, p1, Hp);
        apply_hz(g, &T, q1, Hq);
        for (long p = 0; p < N; p++) {
            const double h0p = Lp[p] - Hp[p];
            rp[p] = E[p] * h0p + S[p] * Hq[p];
            rq[p] = S[p] * h0p + Hq[p];
        }
        if (vol_src)
            for (long p = 0; p < N; p++) {
                rp[p] += vol_src[(2L * n) * N + p];
                rq[p] += vol_src[(2L * n + 1) * N + p];
            }
        for (int s = 0; s < nsrc; s++)
            for (int c = 0; c < snc[s]; c++) {
                rp[sidx[s][c]] += sw[s][c] * wavelet[n];
                rq[sidx[s][c]] += sw[s][c] * wavelet[n];
            }
        leapfrog(N, dt, m, sigma, rp, p1, p0, p2);
        leapfrog(N, dt, m, sigma, rq, q1, q0, q2);
        for (long p = 0; p < N; p++) {
            const double ap = (p2[p] - 2.0 * p1[p] + p0[p]) / (dt * dt) + sigma[p] * (p2[p] - p0[p]) / (2.0 * dt);
            const double aq = (q2[p] - 2.0 * q1[p] + q0[p]) / (dt * dt) + sigma[p] * (q2[p] - q0[p]) / (2.0 * dt);
            if (udd) {
                udd[(2L * n) * N + p] = ap;
                udd[(2L * n + 1) * N + p] = aq;
            }
            if (r > 0 && Pu)
                for (int i = 0; i < r; i++) {
                    Pu[(long)i * N + p] += Q[(long)n * r + i] * ap;
                    Pu[((long)r + i) * N + p] += Q[(long)n * r + i] * aq;
                }
        }
        if (d)
            for (int j = 0; j < nrec; j++) {
                double acc = 0.0;
                for (int c = 0; c < rnc[j]; c++) acc += rw[j][c] * p2[ridx[j][c]];
                d[(long)n * nrec + j] = acc;
            }
        double *t = p0; p0 = p1; p1 = p2; p2 = t;
        t = q0; q0 = q1; q1 = q2; q2 = t;
    }
done:
    free(E); free(S); free(ax); free(ay); free(az); free(T.t); free(T.d); free(T.w);
    free(ridx); free(rw); free(rnc); free(sigma);
    free(p0); free(p1); free(p2); free(q0); free(q1); free(q2);
    free(Lp); free(Hp); free(Hq); free(rp); free(rq);
    return rc;
}

/*
 * TTI adjoint of one shot (transposed block operator).  Residual injected into the
 * p-equation.  Pv is 2*r*N; grad = sum_j (p_tt^j v_p^j + q_tt^j v_q^j) needs udd (nt*2*N);
 * vpt samples v_p and v_q at npt points: vpt[(j*npt + k)*2 + field].
 */
int orc_tti_adjoint(const orc_grid *g, const double *m, const double *eps, const double *delta,
                    const double *theta, const double *phi, int nrec, const double *rec_xyz,
                    const double *res, int r, const double *Q, double *Pv, const double *udd,
                    double *grad, int npt, const double *pt_xyz, double *vpt)
{
    const long N = orc_npoints(g);
    const int nt = g->nt;
    const double dt = g->dt;
    double *E, *S, *ax, *ay, *az;
    tti_setup(g, eps, delta, theta, phi, &E, &S, &ax, &ay, &az);
    tti_work T = {N, malloc(N * sizeof(double)), malloc(N * sizeof(double)),
                  malloc(N * sizeof(double)), ax, ay, az, g->ndim};
    long (*ridx)[8] = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(*ridx));
    double (*rw)[8] = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(*rw));
    int *rnc = calloc((size_t)(nrec > 0 ? nrec : 1), sizeof(int));
    long (*pidx)[8] = calloc((size_t)(npt > 0 ? npt : 1), sizeof(*pidx));
    double (*pw)[8] = calloc((size_t)(npt > 0 ? npt : 1), sizeof(*pw));
    int *pnc = calloc((size_t)(npt > 0 ? npt : 1), sizeof(int));
    double *sigma = malloc(N * sizeof(double));
    double *a2 = calloc(N, sizeof(double)), *a1 = calloc(N, sizeof(double)), *a0 = calloc(N, sizeof(double));
    double *b2 = calloc(N, sizeof(double)), *b1 = calloc(N, sizeof(double)), *b0 = calloc(N, sizeof(double));
    double *e = malloc(N * sizeof(double)), *f = malloc(N * sizeof(double));
    double *Le = malloc(N * sizeof(double)), *He = malloc(N * sizeof(double));
    double *ra = malloc(N * sizeof(double)), *rb = malloc(N * sizeof(double));
    int rc = 0;
    for (int j = 0; j < nrec && !rc; j++)
        if ((rnc[j] = orc_weights(g, rec_xyz + 3 * j, ridx[j], rw[j])) < 0) rc = -1;
    for (int k = 0; k < npt && !rc; k++)
        if ((pnc[k] = orc_weights(g, pt_xyz + 3 * k, pidx[k], pw[k])) < 0) rc = -1;
    if (rc) goto done;
    orc_sponge(g, sigma);
    if (r > 0 && Pv) memset(Pv, 0, (size_t)2 * r * N * sizeof(double));
    if (grad) memset(grad, 0, N * sizeof(double));
    for (int j = nt - 1; j >= 0; j--) {
        for (long p = 0; p < N; p++) {
            e[p] = E[p] * a1[p] + S[p] * b1[p];
            f[p] = S[p] * a1[p] + b1[p];
        }
        laplacian(g, e, Le);
        apply_hz(g, &T, e, He);
        apply_hz(g, &T, f, rb);
        for (long p = 0; p < N; p++) ra[p] = Le[p] - He[p];
        for (int k = 0; k < nrec; k++)
            for (int c = 0; c < rnc[k]; c++) ra[ridx[k][c]] -= rw[k][c] * res[(long)j * nrec + k];
        leapfrog(N, dt, m, sigma, ra, a1, a2, a0);
        leapfrog(N, dt, m, sigma, rb, b1, b2, b0);
        for (long p = 0; p < N; p++) {
            if (r > 0 && Pv)
                for (int i = 0; i < r; i++) {
                    Pv[(long)i * N + p] += Q[(long)j * r + i] * a0[p];
                    Pv[((long)r + i) * N + p] += Q[(long)j * r + i] * b0[p];
                }
            if (grad && udd)
                grad[p] += udd[(2L * j) * N + p] * a0[p] + udd[(2L * j + 1) * N + p] * b0[p];
        }
        for (int k = 0; k < npt; k++) {
            double sa = 0.0, sb = 0.0;
            for (int c = 0; c < pnc[k]; c++) {
                sa += pw[k][c] * a0[pidx[k][c]];
                sb += pw[k][c] * b0[pidx[k][c]];
            }
            vpt[((long)j * npt + k) * 2] = sa;
            vpt[((long)j * npt + k) * 2 + 1] = sb;
        }
        double *t = a2; a2 = a1; a1 = a0; a0 = t;
        t = b2; b2 = b1; b1 = b0; b0 = t;
    }
done:
    free(E); free(S); free(ax); free(ay); free(az); free(T.t); free(T.d); free(T.w);
    free(ridx); free(rw); free(rnc); free(pidx); free(pw); free(pnc); free(sigma);
    free(a2); free(a1); free(a0); free(b2); free(b1); free(b0);
    free(e); free(f); free(Le); free(He); free(ra); free(rb);
    return rc;
}
