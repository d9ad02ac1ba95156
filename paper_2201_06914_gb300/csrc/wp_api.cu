// C ABI of libwp.so (include/wp.h): validation, workspace carving, acquisition tables and
// the time loops of the probed (Eq. 3) and exact (Eq. 2) gradients.  All device work runs
// in the kernels of stencil.cu, probe_gemm.cu and aux.cu; this file only orchestrates.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "wp_internal.cuh"

using namespace wp;

struct wp_model_s {
    wp_model_desc desc;
    GridDev G;
    double vmin, vmax;
    int probe_layout;   // WP_PROBES_DENSE or WP_PROBES_ALIGNED (P_u, P_v of the probed calls)
};

namespace {

thread_local std::string g_err;

wp_status fail(wp_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define WP_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(WP_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                \
    } while (0)

// Leapfrog stability constant of the 8th-order second derivative: the largest eigenvalue
// of -D2 is (205/72 + 2*(8/5 + 1/5 + 8/315 + 1/560)) / h^2.
constexpr double kLambda1D = 205.0 / 72.0 + 2.0 * (8.0 / 5.0 + 1.0 / 5.0 + 8.0 / 315.0 + 1.0 / 560.0);

// Bump allocator over a workspace (or over address 0 to measure one).
struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *b) : base((char *)b) {}
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = (T *)(base + off);
        off += count * sizeof(T);
        return p;
    }
};

// ---------------------------------------------------------------------------------------
// Acquisition tables (host-built, uploaded into the workspace).
// ---------------------------------------------------------------------------------------
int key_count(const GridDev &G) { return (int)stencil_keys(G); }
int ncorner(const GridDev &G) { return G.ndim == 2 ? 4 : 8; }

// Grid corners and bilinear/trilinear weights of a point (metres from the first interior
// point); false when the point is not strictly inside the padded grid.
bool corners(const wp_model_s *M, const double *xyz, int ix[8], int iy[8], int iz[8], double w[8])
{
    const GridDev &G = M->G;
    const double gx = G.nbl + xyz[0] / M->desc.dx, gz = G.nbl + xyz[2] / M->desc.dz;
    const double gy = G.ndim == 3 ? G.nbl + xyz[1] / M->desc.dy : 0.0;
    if (!(gx >= 0 && gx < G.NX - 1 && gz >= 0 && gz < G.NZ - 1)) return false;
    if (G.ndim == 3 && !(gy >= 0 && gy < G.NY - 1)) return false;
    const int bx = (int)floor(gx), by = (int)floor(gy), bz = (int)floor(gz);
    const double fx = gx - bx, fy = gy - by, fz = gz - bz;
    int n = 0;
    for (int cz = 0; cz < 2; cz++)
        for (int cy = 0; cy < (G.ndim == 3 ? 2 : 1); cy++)
            for (int cx = 0; cx < 2; cx++) {
                ix[n] = bx + cx;
                iy[n] = by + cy;
                iz[n] = bz + cz;
                w[n] = (cx ? fx : 1 - fx) * (cz ? fz : 1 - fz) *
                       (G.ndim == 3 ? (cy ? fy : 1 - fy) : 1.0);
                n++;
            }
    return true;
}

struct InjTable {
    std::vector<int> off;
    std::vector<InjEntry> ent;
};

// CSR of injection entries keyed by (shot, stencil tile[, plane]) for npts points per shot.
bool build_injection(const wp_model_s *M, int nshots, int npts, const double *xyz, InjTable &T)
{
    const GridDev &G = M->G;
    const int K = key_count(G), nc = ncorner(G);
    T.off.assign((size_t)nshots * (K + 1), 0);
    T.ent.clear();
    T.ent.reserve((size_t)nshots * npts * nc);
    std::vector<int> keys;
    std::vector<InjEntry> tmp;
    for (int s = 0; s < nshots; s++) {
        keys.clear();
        tmp.clear();
        for (int j = 0; j < npts; j++) {
            int ix[8], iy[8], iz[8];
            double w[8];
            if (!corners(M, xyz + 3 * ((size_t)s * npts + j), ix, iy, iz, w)) return false;
            for (int c = 0; c < nc; c++) {
                InjEntry e;
                const int TX = tile_x(G), TY = tile_y(G);
                const int tile = ix[c] / TX + tiles_x(G) * (iy[c] / TY + tiles_y(G) * (iz[c] / G.tz));
                const int key = tile * G.tz + iz[c] % G.tz;
                e.a = ix[c] % TX + TX * (iy[c] % TY);
                e.b = iz[c];
                e.trace = j;
                e.w = (float)w[c];
                keys.push_back(key);
                tmp.push_back(e);
            }
        }
        int *off = T.off.data() + (size_t)s * (K + 1);
        std::vector<int> cnt(K + 1, 0);
        for (int k : keys) cnt[k + 1]++;
        for (int k = 0; k < K; k++) cnt[k + 1] += cnt[k];
        const int base = (int)T.ent.size();
        T.ent.resize(T.ent.size() + tmp.size());
        std::vector<int> pos(cnt.begin(), cnt.end() - 1);
        for (size_t i = 0; i < tmp.size(); i++) T.ent[base + pos[keys[i]]++] = tmp[i];
        for (int k = 0; k <= K; k++) off[k] = base + cnt[k];
    }
    if (T.ent.empty()) T.ent.push_back(InjEntry{0, 0, 0, 0.f});
    return true;
}

// The same table in the two-step tiling (stencil2.cu): keyed by (shot, tile, plane of the
// segment extended by RAD planes on each side); an entry inside the overlap of two tiles
// or two extended segments is listed under each, with its column offset in that tile.
bool build_injection2(const wp_model_s *M, int nshots, int npts, const double *xyz, InjTable &T)
{
    const GridDev &G = M->G;
    const long long K = stencil2_keys(G);
    const int nc = ncorner(G), C = core2_x(G), TX = G.tx, ntx = tiles2_x(G), nsz = tiles2_z(G);
    const int KP = G.tz2 + 2 * RAD;
    T.off.assign((size_t)nshots * (K + 1), 0);
    T.ent.clear();
    std::vector<long long> keys;
    std::vector<InjEntry> tmp;
    for (int s = 0; s < nshots; s++) {
        keys.clear();
        tmp.clear();
        for (int j = 0; j < npts; j++) {
            int ix[8], iy[8], iz[8];
            double w[8];
            if (!corners(M, xyz + 3 * ((size_t)s * npts + j), ix, iy, iz, w)) return false;
            for (int c = 0; c < nc; c++) {
                for (int t = std::max(0, (ix[c] + RAD) / C - 1); t <= std::min(ntx - 1, (ix[c] + RAD) / C); t++) {
                    const int x0 = t * C - RAD;
                    if (ix[c] < x0 || ix[c] >= x0 + TX) continue;
                    for (int q = std::max(0, (iz[c] - RAD) / G.tz2 - 1); q <= std::min(nsz - 1, (iz[c] + RAD) / G.tz2); q++) {
                        const int z0 = q * G.tz2, z1 = std::min(z0 + G.tz2, G.NZ);
                        if (iz[c] < z0 - RAD || iz[c] >= z1 + RAD) continue;
                        InjEntry e;
                        e.a = ix[c] - x0;
                        e.b = iz[c];
                        e.trace = j;
                        e.w = (float)w[c];
                        keys.push_back((long long)(q * ntx + t) * KP + (iz[c] - (z0 - RAD)));
                        tmp.push_back(e);
                    }
                }
            }
        }
        int *off = T.off.data() + (size_t)s * (K + 1);
        std::vector<int> cnt(K + 1, 0);
        for (long long k : keys) cnt[k + 1]++;
        for (long long k = 0; k < K; k++) cnt[k + 1] += cnt[k];
        const int base = (int)T.ent.size();
        T.ent.resize(T.ent.size() + tmp.size());
        std::vector<int> pos(cnt.begin(), cnt.end() - 1);
        for (size_t i = 0; i < tmp.size(); i++) T.ent[base + pos[keys[i]]++] = tmp[i];
        for (long long k = 0; k <= K; k++) off[k] = base + cnt[k];
    }
    if (T.ent.empty()) T.ent.push_back(InjEntry{0, 0, 0, 0.f});
    return true;
}

bool build_gather(const wp_model_s *M, int nshots, int nrec, const double *xyz,
                  std::vector<int> &idx, std::vector<float> &w)
{
    const GridDev &G = M->G;
    const int nc = ncorner(G);
    idx.assign((size_t)nshots * nrec * nc, 0);
    w.assign((size_t)nshots * nrec * nc, 0.f);
    for (size_t q = 0; q < (size_t)nshots * nrec; q++) {
        int ix[8], iy[8], iz[8];
        double ww[8];
        if (!corners(M, xyz + 3 * q, ix, iy, iz, ww)) return false;
        for (int c = 0; c < nc; c++) {
            idx[q * nc + c] = (iz[c] * G.NY + iy[c]) * G.NXp + ix[c];
            w[q * nc + c] = (float)ww[c];
        }
    }
    return true;
}

size_t inj_ints(const GridDev &G, int nshots) { return (size_t)nshots * (key_count(G) + 1); }

// ---------------------------------------------------------------------------------------
// Workspace layouts.
// ---------------------------------------------------------------------------------------
struct Tables {
    int *src_off = nullptr; InjEntry *src_ent = nullptr;
    int *rec_off = nullptr; InjEntry *rec_ent = nullptr;
    int *g_idx = nullptr; float *g_w = nullptr;   // receiver corners (recording, TTI adjoint)
    double *g_acc = nullptr;                      // u at the receiver corners ((w, d) form)
    int *s_idx = nullptr; float *s_w = nullptr;   // source corners (TTI forward)
    // two-step tiling (2-D isotropic with G.tz2 > 0)
    int *src2_off = nullptr; InjEntry *src2_ent = nullptr;
    int *rec2_off = nullptr; InjEntry *rec2_ent = nullptr;
};

struct Layout {
    int *err = nullptr;
    double *partials = nullptr;
    double *misfit = nullptr;
    float *b = nullptr;
    Tables t;
    // probed
    float *u = nullptr;     // [shot][3][N]: u^n, u^{n+1} and the input of a pending record row
    float *ring = nullptr;  // [shot][Tb+1][ring_stride]
    long long ring_stride = 0;  // N rounded up to 128 floats (512-byte rows)
    float *pv = nullptr;    // internal P_u / P_v: [shot][r][ring_stride], points at pitch NXp
    float *img = nullptr;   // [shot][N]
    __nv_bfloat16 *qhi = nullptr, *qlo = nullptr;  // probe images [shot][block][chunk][r_pad*64]
    // exact
    float *hist = nullptr;  // [shot][slots][N]
    float *ckpt = nullptr;  // [shot][ncp][2][N]
    float *v = nullptr;     // [shot][3][N]  (v0, v1, mu)
    float *dsyn = nullptr, *res = nullptr;
    // TTI: parameter fields (padded) and the Dr scratch per virtual shot
    float *E = nullptr, *Sd = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr;
    float *tscr = nullptr;
    float *ef = nullptr;    // TTI adjoint: [2][virtual shot][N] the combined fields e, f (ping-pong)
    size_t total = 0;
};

int r_pad_of(int r) { return std::max(16, (r + 15) / 16 * 16); }
int nt_pad_of(int nt) { return (nt + 63) / 64 * 64 + 64; }
long long ring_stride_of(long long N) { return (N + 127) / 128 * 128; }
int nblocks_of(int nt, int Tb) { return (nt + Tb - 1) / Tb; }
int ncb_of(int Tb) { return (Tb + 63) / 64; }

Layout make_layout(const wp_model_s *M, const wp_geom *g, int r, int Tb, int mode, void *ws)
{
    Layout L;
    Carve c(ws);
    const long long N = M->G.N, NP = M->G.Np;
    const int S = g->nshots, nt = M->desc.nt, nc = ncorner(M->G);
    const int NF = M->G.tti ? 2 : 1;          // wavefields per shot
    const size_t SV = (size_t)S * NF;         // virtual shots
    const size_t nr = (size_t)S * g->nrec;
    L.err = c.take<int>(64);
    const int nparts = residual_parts((long long)S * nt * g->nrec);
    L.partials = c.take<double>(nparts);
    L.misfit = c.take<double>(1);
    L.b = c.take<float>(NP);
    const size_t ki = inj_ints(M->G, S);
    L.t.src_off = c.take<int>(ki);
    L.t.src_ent = c.take<InjEntry>(std::max<size_t>(1, (size_t)S * g->nsrc * nc));
    L.t.rec_off = c.take<int>(ki);
    L.t.rec_ent = c.take<InjEntry>(std::max<size_t>(1, nr * nc));
    L.t.g_idx = c.take<int>(std::max<size_t>(1, nr * nc));
    L.t.g_w = c.take<float>(std::max<size_t>(1, nr * nc));
    L.t.g_acc = c.take<double>(std::max<size_t>(1, nr * nc));
    if (M->G.tz2 > 0) {   // an entry can fall in two tiles and two extended segments
        const size_t ki2 = (size_t)S * (stencil2_keys(M->G) + 1);
        L.t.src2_off = c.take<int>(ki2);
        L.t.src2_ent = c.take<InjEntry>(std::max<size_t>(1, (size_t)S * g->nsrc * nc * 4));
        L.t.rec2_off = c.take<int>(ki2);
        L.t.rec2_ent = c.take<InjEntry>(std::max<size_t>(1, nr * nc * 4));
    }
    if (M->G.tti) {
        L.t.s_idx = c.take<int>(std::max<size_t>(1, (size_t)S * g->nsrc * nc));
        L.t.s_w = c.take<float>(std::max<size_t>(1, (size_t)S * g->nsrc * nc));
        L.E = c.take<float>(NP);
        L.Sd = c.take<float>(NP);
        L.ax = c.take<float>(NP);
        L.ay = c.take<float>(NP);
        L.az = c.take<float>(NP);
        L.tscr = c.take<float>(SV * NP);
        L.ef = c.take<float>(2 * SV * NP);
    }
    if (mode == WP_MODE_PROBED) {
        const int rp = r_pad_of(r);
        const size_t nimg = (size_t)S * nblocks_of(nt, Tb) * ncb_of(Tb) * rp * 64;
        L.ring_stride = ring_stride_of(NP);
        L.u = c.take<float>(SV * 3 * NP);
        L.ring = c.take<float>(SV * (Tb + 1) * L.ring_stride);
        L.pv = c.take<float>(SV * std::max(r, 1) * L.ring_stride);   // internal P (pitch ring_stride)
        L.img = c.take<float>(SV * N);
        L.qhi = c.take<__nv_bfloat16>(nimg);
        L.qlo = c.take<__nv_bfloat16>(nimg);
    } else {
        const int slots = mode == WP_MODE_EXACT_FULL ? nt + 1 : Tb + 1;
        L.u = c.take<float>(SV * 3 * NP);
        L.hist = c.take<float>(SV * slots * NP);
        if (mode == WP_MODE_EXACT_CHECKPOINT) {
            const int ncp = (nt + Tb - 1) / Tb;
            L.ckpt = c.take<float>(SV * ncp * 2 * NP);
        }
        L.v = c.take<float>(SV * 4 * NP);   // v in two buffers, its increment in two
        L.img = c.take<float>((size_t)S * NP);
        L.dsyn = c.take<float>(std::max<size_t>(1, nr * nt));
        L.res = c.take<float>(std::max<size_t>(1, nr * nt));
    }
    L.total = c.off + 256;
    return L;
}

wp_status check_geom(const wp_model_s *M, const wp_geom *g)
{
    if (!g) return fail(WP_ERR_INVALID, "geometry is NULL");
    if (g->nshots < 1 || g->nsrc < 0 || g->nrec < 0)
        return fail(WP_ERR_INVALID, "need nshots >= 1, nsrc >= 0, nrec >= 0");
    if (g->nsrc > 0 && !g->src_xyz) return fail(WP_ERR_INVALID, "src_xyz is NULL");
    if (g->nrec > 0 && !g->rec_xyz) return fail(WP_ERR_INVALID, "rec_xyz is NULL");
    (void)M;
    return WP_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

template <class T>
wp_status upload(T *dst, const std::vector<T> &src, cudaStream_t s)
{
    if (src.empty()) return WP_OK;
    WP_CUDA(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return WP_OK;
}

wp_status prepare_tables(const wp_model_s *M, const wp_geom *g, const Layout &L, bool src,
                         bool rec_inj, bool gather, cudaStream_t s)
{
    InjTable T;
    if (src) {
        if (!build_injection(M, g->nshots, g->nsrc, g->src_xyz, T))
            return fail(WP_ERR_INVALID, "a source lies outside the padded grid");
        if (upload(L.t.src_off, T.off, s) || upload(L.t.src_ent, T.ent, s)) return WP_ERR_CUDA;
    }
    if (rec_inj) {
        if (!build_injection(M, g->nshots, g->nrec, g->rec_xyz, T))
            return fail(WP_ERR_INVALID, "a receiver lies outside the padded grid");
        if (upload(L.t.rec_off, T.off, s) || upload(L.t.rec_ent, T.ent, s)) return WP_ERR_CUDA;
    }
    if (M->G.tz2 > 0 && src) {
        InjTable T2;
        if (!build_injection2(M, g->nshots, g->nsrc, g->src_xyz, T2))
            return fail(WP_ERR_INVALID, "a source lies outside the padded grid");
        if (upload(L.t.src2_off, T2.off, s) || upload(L.t.src2_ent, T2.ent, s)) return WP_ERR_CUDA;
    }
    if (M->G.tz2 > 0 && rec_inj) {
        InjTable T2;
        if (!build_injection2(M, g->nshots, g->nrec, g->rec_xyz, T2))
            return fail(WP_ERR_INVALID, "a receiver lies outside the padded grid");
        if (upload(L.t.rec2_off, T2.off, s) || upload(L.t.rec2_ent, T2.ent, s)) return WP_ERR_CUDA;
    }
    if (src && M->G.tti && g->nsrc > 0) {
        std::vector<int> idx;
        std::vector<float> w;
        if (!build_gather(M, g->nshots, g->nsrc, g->src_xyz, idx, w))
            return fail(WP_ERR_INVALID, "a source lies outside the padded grid");
        if (upload(L.t.s_idx, idx, s) || upload(L.t.s_w, w, s)) return WP_ERR_CUDA;
    }
    if (gather && g->nrec > 0) {
        std::vector<int> idx;
        std::vector<float> w;
        if (!build_gather(M, g->nshots, g->nrec, g->rec_xyz, idx, w))
            return fail(WP_ERR_INVALID, "a receiver lies outside the padded grid");
        if (upload(L.t.g_idx, idx, s) || upload(L.t.g_w, w, s)) return WP_ERR_CUDA;
    }
    return WP_OK;
}

// Stencil arguments common to every step of one sweep.
StencilArgs base_args(const wp_model_s *M, const wp_geom *g, const Layout &L)
{
    StencilArgs A{};
    A.b = L.b;
    A.err = L.err;
    A.nshots = g->nshots;
    A.nrec = g->nrec;
    A.ncorner = ncorner(M->G);
    A.g_idx = L.t.g_idx;
    A.g_w = L.t.g_w;
    return A;
}

void set_source_injection(StencilArgs &A, const Layout &L, const wp_geom *g, const float *wavelet)
{
    A.inj_off = g->nsrc > 0 ? L.t.src_off : nullptr;
    A.inj = g->nsrc > 0 ? L.t.src_ent : nullptr;
    A.traces = wavelet;
    A.tr_ss = 0;
    A.tr_ts = 1;
    A.tr_rs = 0;
    A.tr_sign = 1.f;
}

void set_residual_injection(StencilArgs &A, const Layout &L, const wp_geom *g, const float *res,
                            int nt)
{
    A.inj_off = g->nrec > 0 ? L.t.rec_off : nullptr;
    A.inj = g->nrec > 0 ? L.t.rec_ent : nullptr;
    A.traces = res;
    A.tr_ss = (long long)nt * g->nrec;
    A.tr_ts = g->nrec;
    A.tr_rs = 1;
    A.tr_sign = -1.f;
}

wp_status common_checks(const wp_model_s *M, const wp_geom *g)
{
    if (!M) return fail(WP_ERR_INVALID, "model is NULL");
    return check_geom(M, g);
}

// One time step of every shot: the isotropic tiled stencil, or the three TTI launches.
// `adjoint` selects the transposed TTI operator and the receiver-side injection.
wp_status launch_step(const wp_model_s *M, const wp_geom *g, const Layout &L, const StencilArgs &A,
                      bool imaging, bool adjoint, cudaStream_t s)
{
    if (!M->G.tti) {
        WP_CUDA(launch_stencil(M->G, A, imaging, s));
        return WP_OK;
    }
    TtiArgs T{};
    T.u_in = A.u_in; T.u_in_ss = A.u_in_ss;
    T.d_in = A.d_in; T.d_in_ss = A.d_in_ss;
    T.u_out = A.u_out; T.u_out_ss = A.u_out_ss;
    T.d_out = A.d_out; T.d_out_ss = A.d_out_ss;
    T.b = L.b;
    T.E = L.E; T.Sd = L.Sd; T.ax = L.ax; T.ay = L.ay; T.az = L.az;
    T.t = L.tscr; T.t_ss = M->G.Np;
    T.err = L.err;
    T.adjoint = adjoint ? 1 : 0;
    if (adjoint) {   // step j reads e, f of step j+1 and writes its own
        const size_t SVN = (size_t)g->nshots * 2 * M->G.Np;
        T.ef_in = L.ef + (size_t)((A.step + 1) & 1) * SVN;
        T.ef_out = L.ef + (size_t)(A.step & 1) * SVN;
        T.ef_ss = M->G.Np;
    }
    if (imaging) {
        T.img = A.img; T.img_ss = A.img_ss;
        T.h1 = A.h1; T.h0 = A.h0; T.h_ss = A.h_ss; T.img_scale = A.img_scale;
    }
    T.nshots = g->nshots;
    TtiInject J{};
    J.ncorner = ncorner(M->G);
    J.traces = A.traces; J.tr_ss = A.tr_ss; J.tr_ts = A.tr_ts; J.tr_rs = A.tr_rs;
    J.step = A.step; J.sign = A.tr_sign;
    if (!adjoint) {
        J.idx = L.t.s_idx; J.w = L.t.s_w; J.npts = g->nsrc; J.both = 1;
    } else {
        J.idx = L.t.g_idx; J.w = L.t.g_w; J.npts = g->nrec; J.both = 0;
    }
    WP_CUDA(launch_tti_step(M->G, T, J, s));
    if (A.do_gather) {
        StencilArgs Gq = A;
        Gq.u_in_ss = 2 * A.u_in_ss;   // record field p (virtual shot 2s)
        WP_CUDA(launch_gather(M->G, Gq, s));
    }
    return WP_OK;
}

// Forward sweep that records d (row n = R u^{n+1}) and writes increments into `dring`
// (nslots slots per shot, slot = n mod nslots; nslots = 1 keeps a single increment).
// `ckpt` (or NULL) receives the state entering step n for n a multiple of `cint`: (w^{n-1},
// d^n) in the (w, d) form of the isotropic equation, (u^n, d^n) for TTI.  `on_step(n)` runs
// after the launch that completes step n.  On 2-D isotropic grids steps n and n+1 share
// one two-step launch when `pairable(n)` says that on_step(n) has nothing to do, no
// checkpoint falls at n+1 and the ring keeps d^{n+1} until the next launch has recorded
// row n from it (nslots >= 4).
//
// Isotropic grids march the (w, d) form: the increments are the stencil field and live in
// the ring (launch n reads slot n and writes slot n+1, a pair also slot n+2), w = L u
// alternates between two buffers per shot, and u at the receiver corners accumulates in
// FP64 in the recording blocks.  TTI marches (u, d) with three u buffers per shot (u^n, the
// output, and the input of the previous pair while its first row is pending).
template <class F, class P>
wp_status forward_sweep(const wp_model_s *M, const wp_geom *g, const Layout &L,
                        const float *wavelet, float *d_out, float *dring, int nslots,
                        long long sstride, float *ckpt, int cint, cudaStream_t s, F on_step,
                        P pairable)
{
    const long long N = M->G.Np;  // internal (padded) field size
    const int S = g->nshots * (M->G.tti ? 2 : 1), nt = M->desc.nt;   // virtual shots
    const bool wd = !M->G.tti;
    WP_CUDA(launch_fill(L.u, (long long)S * 3 * N, 0.f, s));
    WP_CUDA(cudaMemset2DAsync(dring, (size_t)nslots * sstride * sizeof(float), 0, N * sizeof(float), S, s));
    StencilArgs A = base_args(M, g, L);
    set_source_injection(A, L, g, wavelet);
    const int *off1 = A.inj_off;
    const InjEntry *ent1 = A.inj;
    const int *off2 = g->nsrc > 0 ? L.t.src2_off : nullptr;
    const InjEntry *ent2 = g->nsrc > 0 ? L.t.src2_ent : nullptr;
    const long long ring_ss = (long long)nslots * sstride;
    if (wd) {
        A.wd = 1;
        A.u_in_ss = A.u_out_ss = A.u1_ss = A.gp_d_ss = ring_ss;
        A.d_in_ss = A.d_out_ss = 3 * N;
        A.g_acc = L.t.g_acc;
        if (d_out && g->nrec > 0)
            WP_CUDA(cudaMemsetAsync(L.t.g_acc, 0, (size_t)g->nshots * g->nrec * ncorner(M->G) * sizeof(double), s));
    } else {
        A.u_in_ss = A.u_out_ss = A.gp_u_ss = 3 * N;
        A.d_in_ss = A.d_out_ss = A.d1_ss = A.gp_d_ss = ring_ss;
    }
    A.g_out = d_out;
    A.g_ss = (long long)nt * g->nrec;
    const bool rec = d_out && g->nrec > 0;
    const bool two_ok = M->G.tz2 > 0 && !M->G.tti && nslots >= 4;
    auto ubuf = [&](int k) { return L.u + (size_t)k * N; };
    auto slot = [&](int n) { return dring + (size_t)(n % nslots) * sstride; };
    int cur = 0, pend = -1, pend_row = -1;
    for (int n = 0; n < nt;) {
        if (ckpt && n % cint == 0) {
            float *cp = ckpt + (size_t)(n / cint) * 2 * N;
            const size_t ncp = (nt + cint - 1) / cint;
            WP_CUDA(cudaMemcpy2DAsync(cp, ncp * 2 * N * sizeof(float), ubuf(cur), 3 * N * sizeof(float),
                                      N * sizeof(float), S, cudaMemcpyDeviceToDevice, s));
            WP_CUDA(cudaMemcpy2DAsync(cp + N, ncp * 2 * N * sizeof(float), slot(n),
                                      (size_t)nslots * sstride * sizeof(float), N * sizeof(float), S,
                                      cudaMemcpyDeviceToDevice, s));
        }
        const bool two = two_ok && n + 1 < nt && pairable(n) && !(ckpt && (n + 1) % cint == 0);
        int out = 0;
        if (wd) out = cur ^ 1;   // w ping-pong (a pair must not overwrite w^{n-1} in place)
        else
            while (out == cur || out == pend) out++;
        A.step = n;
        A.do_gather = (rec && n >= 1) ? 1 : 0;
        A.g_row = n - 1;
        A.do_pend = (rec && pend >= 0) ? 1 : 0;
        if (pend >= 0) {
            A.gp_u = ubuf(pend);
            A.gp_d = slot(pend_row + 1);
            A.gp_row = pend_row;
        }
        if (wd) {
            A.u_in = slot(n);       // d^n
            A.d_in = ubuf(cur);     // w^{n-1}
            A.d_out = ubuf(out);    // w^n (w^{n+1} for a pair)
        } else {
            A.u_in = ubuf(cur);
            A.u_out = ubuf(out);
            A.d_in = slot(n);
        }
        wp_status st;
        if (two) {
            A.inj_off = off2;
            A.inj = ent2;
            if (wd) {
                A.u1_out = slot(n + 1);
                A.d1_out = nullptr;
                A.u_out = slot(n + 2);
            } else {
                A.d1_out = slot(n + 1);
                A.u1_out = nullptr;
                A.d_out = slot(n + 2);
            }
            A.step2 = n + 1;
            WP_CUDA(launch_stencil2(M->G, A, s));
            if ((st = on_step(n)) != WP_OK || (st = on_step(n + 1)) != WP_OK) return st;
            pend = cur;
            pend_row = n;
            cur = out;
            n += 2;
        } else {
            A.inj_off = off1;
            A.inj = ent1;
            if (wd) A.u_out = slot(n + 1);
            else A.d_out = slot(n + 1);
            if ((st = launch_step(M, g, L, A, false, false, s)) != WP_OK) return st;
            if ((st = on_step(n)) != WP_OK) return st;
            pend = -1;
            cur = out;
            n += 1;
        }
    }
    if (rec) {
        A.u_in = wd ? slot(nt) : ubuf(cur);
        A.g_row = nt - 1;
        A.do_gather = 1;
        A.do_pend = pend >= 0 ? 1 : 0;
        if (pend >= 0) {
            A.gp_u = ubuf(pend);
            A.gp_d = slot(pend_row + 1);
            A.gp_row = pend_row;
        }
        if (M->G.tti) A.u_in_ss *= 2;   // record field p
        WP_CUDA(launch_gather(M->G, A, s));
    }
    return WP_OK;
}

wp_status prepare_tti(const wp_model_s *M, const Layout &L, cudaStream_t s)
{
    if (!M->G.tti) return WP_OK;
    WP_CUDA(launch_tti_params(M->G, M->desc.eps, M->desc.delta, M->desc.theta, M->desc.phi, L.E,
                              L.Sd, L.ax, L.ay, L.az, s));
    return WP_OK;
}

PipeArgs pipe_base(const wp_model_s *M, const Layout &L, int r, int Tb)
{
    PipeArgs P{};
    P.ring = L.ring;
    P.sstride = L.ring_stride;
    P.N = M->G.N;
    P.Np = M->G.Np;
    P.NX = M->G.NX;
    P.NXp = M->G.NXp;
    P.ntiles = (int)((M->G.Np + 127) / 128);
    P.img_hi = L.qhi;
    P.img_lo = L.qlo;
    P.qlo_nz = L.err + 32;   // set by launch_probe_images (err[0] is the error flag)
    P.nblocks = nblocks_of(M->desc.nt, Tb);
    P.ncb = ncb_of(Tb);
    P.r = r;
    P.r_pad = r_pad_of(r);
    P.img_ld = (long long)P.r_pad * 64;
    P.G = M->G;
    P.err = L.err;
    P.img_div = M->G.tti ? 2 : 1;
    return P;
}

// Per-device resources of model validation: 16 floats of static device memory and a
// non-blocking stream (created once per device, kept for the life of the process).
__device__ float g_validation_scratch[16];
std::mutex g_val_mtx;
cudaStream_t g_val_stream[64] = {};
float *g_val_ptr[64] = {};

cudaError_t validation_resources(float **scratch, cudaStream_t *stream)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_val_mtx);
    if (!g_val_stream[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_validation_scratch);
        if (e != cudaSuccess) return e;
        e = cudaStreamCreateWithFlags(&g_val_stream[dev], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        g_val_ptr[dev] = (float *)p;
    }
    *scratch = g_val_ptr[dev];
    *stream = g_val_stream[dev];
    return cudaSuccess;
}

// Planes marched by one stencil block.  Short marches give more blocks (about eight waves
// of resident blocks balance the uneven blocks: injection, absorbing layers, the ragged
// last segment, the prologue latency); long marches amortise the 8-plane z halo, so the
// march is kept >= 24 planes where the grid allows.
int choose_tz(const GridDev &G, int nshots)
{
    if (const char *e = getenv("WP_STENCIL_TZ")) {
        const int v = atoi(e);
        if (v >= 1) return std::min(v, G.NZ);
    }
    const long long cols = (long long)tiles_x(G) * tiles_y(G) * nshots;
    const long long cap = (long long)device_sm_count() * stencil_blocks_per_sm(G);
    const long long segs = std::max<long long>(1, (8 * cap + cols - 1) / cols);
    int tz = (int)((G.NZ + segs - 1) / segs);
    tz = std::max(tz, std::min(24, G.NZ));
    const int nseg = (G.NZ + tz - 1) / tz;
    return (G.NZ + nseg - 1) / nseg;   // equal segments
}

// Planes per two-step segment (2-D isotropic grids; 0 turns two-step launches off).  A
// segment recomputes 8 planes of its first step (4 beyond either end), so segments are
// kept at >= 32 planes; otherwise they are sized for about four waves of resident blocks
// (on the 64-shot 1601 x 401 model: 8 segments of 61 planes, measured fastest among
// 25..121 planes).
int choose_tz2(const GridDev &G, int nshots)
{
    if (G.ndim != 2 || G.tti) return 0;
    if (const char *e = getenv("WP_STENCIL2"))
        if (atoi(e) == 0) return 0;
    if (const char *e = getenv("WP_STENCIL2_TZ")) {
        const int v = atoi(e);
        if (v >= 1) return std::min(v, G.NZ);
    }
    const long long cap = (long long)device_sm_count() * stencil2_blocks_per_sm(G);
    const long long cols = (long long)tiles2_x(G) * nshots;
    const long long segs = std::max<long long>(1, (4 * cap + cols / 2) / cols);
    int tz = (int)((G.NZ + segs - 1) / segs);
    tz = std::max(tz, std::min(32, G.NZ));
    const int nseg = (G.NZ + tz - 1) / tz;
    return (G.NZ + nseg - 1) / nseg;   // equal segments
}

// The model as one call sees it: the march lengths depend on the batch size.
wp_model_s call_model(const wp_model_s *M, const wp_geom *g)
{
    wp_model_s C = *M;
    const int ns = g ? std::max(1, g->nshots) : 1;
    C.G.tz = choose_tz(C.G, ns);
    C.G.tz2 = choose_tz2(C.G, ns);
    return C;
}

}  // namespace

void wp::set_last_error(const char *msg) { g_err = msg; }

// =======================================================================================
// C ABI
// =======================================================================================
extern "C" {

const char *wp_last_error(void) { return g_err.c_str(); }

long long wp_kernel_launches(void) { return launches(); }

wp_status wp_model(const wp_model_desc *d, wp_model_t **out)
{
    if (!d || !out) return fail(WP_ERR_INVALID, "desc/out is NULL");
    *out = nullptr;
    if (d->ndim != 2 && d->ndim != 3) return fail(WP_ERR_INVALID, "ndim must be 2 or 3");
    if (d->space_order != 8) return fail(WP_ERR_INVALID, "space_order must be 8");
    if (d->physics != WP_PHYS_ISO && d->physics != WP_PHYS_TTI)
        return fail(WP_ERR_INVALID, "physics must be WP_PHYS_ISO or WP_PHYS_TTI");
    if (d->physics == WP_PHYS_TTI && (!d->eps || !d->delta || !d->theta || (d->ndim == 3 && !d->phi)))
        return fail(WP_ERR_INVALID, "TTI needs eps, delta, theta (and phi in 3-D)");
    if (d->nx < 1 || d->nz < 1 || (d->ndim == 3 && d->ny < 1) || d->nbl < 4 || d->nt < 1)
        return fail(WP_ERR_INVALID, "need nx, nz (, ny) >= 1, nbl >= 4, nt >= 1");
    if (!(d->dx > 0) || !(d->dz > 0) || (d->ndim == 3 && !(d->dy > 0)) || !(d->dt > 0))
        return fail(WP_ERR_INVALID, "spacing and dt must be positive");
    if (!d->m || !aligned16(d->m)) return fail(WP_ERR_INVALID, "m must be a 16-byte aligned device pointer");
    GridDev G{};
    G.ndim = d->ndim;
    G.nx = d->nx;
    G.ny = d->ndim == 3 ? d->ny : 1;
    G.nz = d->nz;
    G.nbl = d->nbl;
    G.NX = d->nx + 2 * d->nbl;
    G.NY = d->ndim == 3 ? d->ny + 2 * d->nbl : 1;
    G.NZ = d->nz + 2 * d->nbl;
    G.N = (long long)G.NX * G.NY * G.NZ;
    G.NXp = (G.NX + 3) / 4 * 4;
    G.Np = (long long)G.NXp * G.NY * G.NZ;
    if (G.Np >= (1LL << 31)) return fail(WP_ERR_INVALID, "padded grid must have < 2^31 points");
    G.ihx2 = (float)(1.0 / (d->dx * d->dx));
    G.ihz2 = (float)(1.0 / (d->dz * d->dz));
    G.ihy2 = d->ndim == 3 ? (float)(1.0 / (d->dy * d->dy)) : 0.f;
    G.lrz = (float)((d->dx * d->dx) / (d->dz * d->dz));
    G.lry = d->ndim == 3 ? (float)((d->dx * d->dx) / (d->dy * d->dy)) : 0.f;
    G.lapK = 2.f * (1.f + G.lrz + G.lry);
    G.inv_nbl = 1.f / (float)d->nbl;
    G.tx = stencil_choose_tx(G);
    G.tz = 32;
    G.hx = (float)d->dx;
    G.hy = d->ndim == 3 ? (float)d->dy : 1.f;
    G.hz = (float)d->dz;
    G.tti = d->physics == WP_PHYS_TTI ? 1 : 0;

    // Validate m on the device: positivity, finiteness, velocity range.  The reduction
    // runs on a non-blocking stream of this library with a small static device buffer, so
    // creating a model never synchronises other streams (no cudaMalloc/cudaFree).
    float *scratch = nullptr;
    cudaStream_t vs = nullptr;
    cudaError_t e = validation_resources(&scratch, &vs);
    float init[2] = {3.4e38f, 0.f};
    int zero = 0;
    float mm[2];
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(scratch, init, sizeof init, cudaMemcpyHostToDevice, vs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + 2, &zero, sizeof zero, cudaMemcpyHostToDevice, vs);
    if (e == cudaSuccess) e = launch_minmax(d->m, G.N, scratch, (int *)(scratch + 2), vs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mm, scratch, sizeof mm, cudaMemcpyDeviceToHost, vs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, scratch + 2, sizeof bad, cudaMemcpyDeviceToHost, vs);
    float epsmax = 0.f;
    int delta_gt = 0;
    if (e == cudaSuccess && G.tti) {
        // The anisotropic operator is stiffer by (1 + 2 eps) along the fast direction.
        e = cudaMemsetAsync(scratch + 4, 0, 2 * sizeof(float), vs);
        if (e == cudaSuccess) e = launch_maxval(d->eps, G.N, scratch + 4, vs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&epsmax, scratch + 4, sizeof(float), cudaMemcpyDeviceToHost, vs);
        // where delta > eps the two-field system's symbol has a negative eigenvalue
        // (determinant 2 (eps - delta) |k_perp|^2 |k_par|^2): a growing mode
        if (e == cudaSuccess) e = launch_count_greater(d->delta, d->eps, G.N, (int *)(scratch + 5), vs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&delta_gt, scratch + 5, sizeof(int), cudaMemcpyDeviceToHost, vs);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(vs);
    if (e != cudaSuccess) return fail(WP_ERR_CUDA, "model validation: %s", cudaGetErrorString(e));
    if (bad > 0) return fail(WP_ERR_NONFINITE, "m has %d non-positive or non-finite values", bad);
    if (delta_gt > 0)
        return fail(WP_ERR_UNSTABLE, "delta > eps (or a non-finite Thomsen value) at %d points: the "
                    "pseudo-acoustic TTI system grows without bound there", delta_gt);
    const double vmax = sqrt(1.0 + 2.0 * epsmax) / sqrt((double)mm[0]);
    const double vmin = 1.0 / sqrt((double)mm[1]);
    double ih = 1.0 / (d->dx * d->dx) + 1.0 / (d->dz * d->dz);
    if (d->ndim == 3) ih += 1.0 / (d->dy * d->dy);
    const double lhs = d->dt * d->dt * vmax * vmax * kLambda1D * ih;
    if (lhs > 4.0)
        return fail(WP_ERR_UNSTABLE, "dt=%g exceeds the stability limit %g for v_max=%g", d->dt,
                    2.0 / (vmax * sqrt(kLambda1D * ih)), vmax);
    const double dv = d->damp_v > 0 ? d->damp_v : vmax;
    const double l1000 = log(1000.0);
    G.hs0x = (float)(3.0 * dv * l1000 / (2.0 * d->nbl * d->dx) * d->dt * 0.5);
    G.hs0z = (float)(3.0 * dv * l1000 / (2.0 * d->nbl * d->dz) * d->dt * 0.5);
    G.hs0y = d->ndim == 3 ? (float)(3.0 * dv * l1000 / (2.0 * d->nbl * d->dy) * d->dt * 0.5) : 0.f;
    wp_model_s *M = new wp_model_s;
    M->desc = *d;
    M->desc.damp_v = dv;
    M->G = G;
    M->vmin = vmin;
    M->vmax = vmax;
    M->probe_layout = WP_PROBES_DENSE;
    *out = M;
    return WP_OK;
}

void wp_model_free(wp_model_t *model) { delete model; }

long long wp_model_npoints(const wp_model_t *model) { return model ? model->G.N : -1; }

double wp_model_vmax(const wp_model_t *model) { return model ? model->vmax : 0.0; }

wp_status wp_set_probe_layout(wp_model_t *model, int layout)
{
    if (!model) return fail(WP_ERR_INVALID, "model is NULL");
    if (layout != WP_PROBES_DENSE && layout != WP_PROBES_ALIGNED)
        return fail(WP_ERR_INVALID, "layout must be WP_PROBES_DENSE or WP_PROBES_ALIGNED");
    model->probe_layout = layout;
    return WP_OK;
}

wp_status wp_probe_layout(const wp_model_t *model, int *layout, long long *row_floats, int *x_pitch)
{
    if (!model) return fail(WP_ERR_INVALID, "model is NULL");
    const bool al = model->probe_layout == WP_PROBES_ALIGNED;
    if (layout) *layout = model->probe_layout;
    if (row_floats) *row_floats = al ? ring_stride_of(model->G.Np) : model->G.N;
    if (x_pitch) *x_pitch = al ? model->G.NXp : model->G.NX;
    return WP_OK;
}

size_t wp_workspace_bytes(const wp_model_t *Min, const wp_geom *g, int r, int Tb, int mode)
{
    if (!Min || !g || g->nshots < 1 || r < 0 || r > 512) return 0;
    const wp_model_s MC = call_model(Min, g);
    const wp_model_s *M = &MC;
    if (mode == WP_MODE_PROBED && (Tb < 16 || Tb % 16)) return 0;
    if (mode == WP_MODE_EXACT_CHECKPOINT && Tb < 1) return 0;
    if (mode < 0 || mode > 2) return 0;
    return make_layout(M, g, r, Tb, mode, nullptr).total;
}

wp_status wp_probe_forward(wp_model_t *Min, const wp_geom *g, const float *wavelet, const float *Q,
                           int r, int Tb, float *P_u, float *d_syn, void *ws, size_t ws_bytes,
                           wp_stream stream)
{
    wp_status st = common_checks(Min, g);
    if (st) return st;
    const wp_model_s MC = call_model(Min, g);
    const wp_model_s *M = &MC;
    if (r < 0 || r > 512) return fail(WP_ERR_INVALID, "r must be in 0..512");
    if (Tb < 16 || Tb % 16) return fail(WP_ERR_INVALID, "Tb must be a positive multiple of 16");
    if (!wavelet || (r > 0 && (!Q || !P_u)))
        return fail(WP_ERR_INVALID, "wavelet, Q and P_u are required");
    if (!ws || !aligned16(ws) || (P_u && !aligned16(P_u)) || (Q && !aligned16(Q)))
        return fail(WP_ERR_INVALID, "device pointers must be 16-byte aligned");
    Layout L = make_layout(M, g, r, Tb, WP_MODE_PROBED, ws);
    if (ws_bytes < L.total)
        return fail(WP_ERR_OOM, "workspace %zu < %zu bytes", ws_bytes, L.total);
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = M->G.N;
    const int S = g->nshots, nt = M->desc.nt;
    const int SV = S * (M->G.tti ? 2 : 1);   // virtual shots (TTI: two fields per shot)
    const bool aligned = M->probe_layout == WP_PROBES_ALIGNED;
    if ((st = prepare_tables(M, g, L, true, false, d_syn != nullptr, s))) return st;
    WP_CUDA(cudaMemsetAsync(L.err, 0, 64 * sizeof(int), s));
    WP_CUDA(launch_b_field(M->desc.m, M->desc.dt * M->desc.dt, M->G, L.b, s));
    if ((st = prepare_tti(M, L, s))) return st;
    PipeArgs G = pipe_base(M, L, r, Tb);
    if (r > 0) {
        WP_CUDA(launch_probe_images(Q, S, nt, r, G.r_pad, 0, Tb, G.nblocks, L.qhi, L.qlo, L.err + 32, s));
        G.ring_ss = (long long)(Tb + 1) * L.ring_stride;
        G.nslots = Tb + 1;
        G.mode = 1;
        // accumulated in the row-aligned layout: in P_u itself when the caller asked for
        // that layout, else in the workspace and copied to the dense P_u at the end
        G.P = aligned ? P_u : L.pv;
        G.P_pitch = L.ring_stride;
        G.P_ss = (long long)r * L.ring_stride;
        G.scale = (float)(1.0 / (M->desc.dt * M->desc.dt));
    }
    auto on_step = [&](int n) -> wp_status {
        if (r > 0 && ((n + 1) % Tb == 0 || n == nt - 1)) {
            const int t0 = n / Tb * Tb;
            G.cnt = n + 1 - t0;
            G.slot0 = t0 % (Tb + 1);
            G.blk = t0 / Tb;
            G.p_zero = t0 == 0;   // the first block writes P_u without reading it
            WP_CUDA(launch_probe_pipe(G, SV, s));
        }
        return WP_OK;
    };
    auto pairable = [&](int n) { return !(r > 0 && ((n + 1) % Tb == 0 || n == nt - 1)); };
    st = forward_sweep(M, g, L, wavelet, d_syn, L.ring, Tb + 1, L.ring_stride, nullptr, 1, s, on_step,
                       pairable);
    if (st || r == 0 || aligned) return st;
    WP_CUDA(launch_p_to_user(L.pv, L.ring_stride, (long long)SV * r, N, M->G.NX, M->G.NXp, P_u, s));
    return WP_OK;
}

wp_status wp_adjoint_image(wp_model_t *Min, const wp_geom *g, const float *residual, const float *Q,
                           int r, int Tb, float scale, const float *P_u, float *grad, float *P_v,
                           void *ws, size_t ws_bytes, wp_stream stream)
{
    wp_status st = common_checks(Min, g);
    if (st) return st;
    const wp_model_s MC = call_model(Min, g);
    const wp_model_s *M = &MC;
    if (r < 1 || r > 512) return fail(WP_ERR_INVALID, "r must be in 1..512");
    if (Tb < 16 || Tb % 16) return fail(WP_ERR_INVALID, "Tb must be a positive multiple of 16");
    if (!Q || !P_u || !grad || (g->nrec > 0 && !residual))
        return fail(WP_ERR_INVALID, "residual, Q, P_u and g are required");
    if (!ws || !aligned16(ws) || !aligned16(P_u) || !aligned16(Q) || (P_v && !aligned16(P_v)))
        return fail(WP_ERR_INVALID, "device pointers must be 16-byte aligned");
    Layout L = make_layout(M, g, r, Tb, WP_MODE_PROBED, ws);
    if (ws_bytes < L.total)
        return fail(WP_ERR_OOM, "workspace %zu < %zu bytes", ws_bytes, L.total);
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = M->G.N, NP = M->G.Np;
    const int S = g->nshots, nt = M->desc.nt;
    const int SV = S * (M->G.tti ? 2 : 1);   // virtual shots (TTI: two fields per shot)
    if ((st = prepare_tables(M, g, L, false, true, M->G.tti != 0, s))) return st;
    WP_CUDA(cudaMemsetAsync(L.err, 0, 64 * sizeof(int), s));
    WP_CUDA(launch_b_field(M->desc.m, M->desc.dt * M->desc.dt, M->G, L.b, s));
    if ((st = prepare_tti(M, L, s))) return st;
    // P_v accumulates in the row-aligned layout: in P_v itself when the caller asked for
    // that layout, else in the workspace (copied to a dense P_v at the end if asked for)
    const bool aligned = M->probe_layout == WP_PROBES_ALIGNED;
    float *pv = aligned && P_v ? P_v : L.pv;
    float *mu = L.u;  // [shot][3N]: the increment, ping-pong over the first two N
    WP_CUDA(launch_fill(L.u, (long long)SV * 3 * NP, 0.f, s));
    if (M->G.tti) WP_CUDA(launch_fill(L.ef, (long long)2 * SV * NP, 0.f, s));
    const long long RS = L.ring_stride;
    WP_CUDA(cudaMemset2DAsync(L.ring + (size_t)(nt % Tb) * RS, (size_t)(Tb + 1) * RS * sizeof(float),
                              0, NP * sizeof(float), SV, s));
    PipeArgs G = pipe_base(M, L, r, Tb);
    WP_CUDA(launch_probe_images(Q, S, nt, r, G.r_pad, 0, Tb, G.nblocks, L.qhi, L.qlo, L.err + 32, s));
    G.ring_ss = (long long)(Tb + 1) * RS;
    G.nslots = Tb;
    G.mode = 0;
    G.P = pv;
    G.P_pitch = L.ring_stride;
    G.P_ss = (long long)r * L.ring_stride;
    G.scale = 1.f;

    StencilArgs A = base_args(M, g, L);
    set_residual_injection(A, L, g, residual, nt);
    const int *off1 = A.inj_off;
    const InjEntry *ent1 = A.inj;
    const int *off2 = g->nrec > 0 ? L.t.rec2_off : nullptr;
    const InjEntry *ent2 = g->nrec > 0 ? L.t.rec2_ent : nullptr;
    A.u_in_ss = A.u_out_ss = A.u1_ss = (long long)(Tb + 1) * RS;
    A.d_in_ss = A.d_out_ss = 3 * NP;
    const bool two_ok = M->G.tz2 > 0 && !M->G.tti;
    int dc = 0;
    for (int j = nt - 1; j >= 0;) {
        // a pair (j, j-1) needs no contraction between its steps
        const bool two = two_ok && j >= 1 && j % Tb != 0;
        A.u_in = L.ring + (size_t)((j + 1) % Tb) * RS;
        A.d_in = mu + (size_t)dc * NP;
        A.step = j;
        if (two) {
            A.inj_off = off2;
            A.inj = ent2;
            A.u1_out = L.ring + (size_t)(j % Tb) * RS;
            A.d1_out = nullptr;
            A.u_out = L.ring + (size_t)((j - 1) % Tb) * RS;
            A.d_out = mu + (size_t)(dc ^ 1) * NP;
            A.step2 = j - 1;
            WP_CUDA(launch_stencil2(M->G, A, s));
            dc ^= 1;
            j -= 2;
        } else {
            A.inj_off = off1;
            A.inj = ent1;
            A.u_out = L.ring + (size_t)(j % Tb) * RS;
            A.d_out = mu + (size_t)dc * NP;   // a single step updates the increment in place
            if ((st = launch_step(M, g, L, A, false, true, s))) return st;
            j -= 1;
        }
        const int jd = j + 1;   // the last step done
        if (jd % Tb == 0) {
            G.cnt = std::min(Tb, nt - jd);
            G.slot0 = jd % Tb;
            G.blk = jd / Tb;
            G.p_zero = jd + Tb >= nt;   // the first adjoint block writes P_v without reading it
            WP_CUDA(launch_probe_pipe(G, SV, s));
        }
    }
    // randomized imaging condition (Eq. 3), summed over the (virtual) shots
    WP_CUDA(launch_probe_dot(P_u, aligned, pv, N, M->G.NX, M->G.NXp, L.ring_stride, r, SV, scale, grad, s));
    if (P_v && !aligned)
        WP_CUDA(launch_p_to_user(pv, L.ring_stride, (long long)SV * r, N, M->G.NX, M->G.NXp, P_v, s));
    return WP_OK;
}

wp_status wp_exact_gradient(wp_model_t *Min, const wp_geom *g, const float *wavelet,
                            const float *d_obs, float *grad, double *misfit, float *d_syn, int mode,
                            int ncheck, void *ws, size_t ws_bytes, wp_stream stream)
{
    wp_status st = common_checks(Min, g);
    if (st) return st;
    const wp_model_s MC = call_model(Min, g);
    const wp_model_s *M = &MC;
    if (mode != WP_MODE_EXACT_FULL && mode != WP_MODE_EXACT_CHECKPOINT)
        return fail(WP_ERR_INVALID, "mode must be WP_MODE_EXACT_FULL or WP_MODE_EXACT_CHECKPOINT");
    if (mode == WP_MODE_EXACT_CHECKPOINT && ncheck < 1)
        return fail(WP_ERR_INVALID, "ncheck must be >= 1");
    if (!wavelet || !grad || (g->nrec > 0 && !d_obs))
        return fail(WP_ERR_INVALID, "wavelet, d_obs and g are required");
    if (!ws || !aligned16(ws)) return fail(WP_ERR_INVALID, "workspace must be 16-byte aligned");
    const int cint = mode == WP_MODE_EXACT_CHECKPOINT ? ncheck : 1;
    Layout L = make_layout(M, g, 0, cint, mode, ws);
    if (ws_bytes < L.total)
        return fail(WP_ERR_OOM, "workspace %zu < %zu bytes", ws_bytes, L.total);
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = M->G.Np;  // internal (padded) field size
    const int S = g->nshots, nt = M->desc.nt;
    const int SV = S * (M->G.tti ? 2 : 1);   // virtual shots (TTI: two fields per shot)
    const long long nd = (long long)S * nt * g->nrec;
    if ((st = prepare_tables(M, g, L, true, true, true, s))) return st;
    WP_CUDA(cudaMemsetAsync(L.err, 0, 64 * sizeof(int), s));
    WP_CUDA(launch_b_field(M->desc.m, M->desc.dt * M->desc.dt, M->G, L.b, s));
    if ((st = prepare_tti(M, L, s))) return st;
    float *dsyn = d_syn ? d_syn : L.dsyn;
    const bool full = mode == WP_MODE_EXACT_FULL;
    const int hslots = full ? nt + 1 : cint + 1;
    const float inv_dt2 = (float)(1.0 / (M->desc.dt * M->desc.dt));
    auto nop = [](int) { return WP_OK; };
    // Forward: full history of increments, or one increment plus checkpoints.
    auto any = [](int) { return true; };
    if (full) st = forward_sweep(M, g, L, wavelet, dsyn, L.hist, hslots, N, nullptr, 1, s, nop, any);
    else st = forward_sweep(M, g, L, wavelet, dsyn, L.hist, hslots, N, L.ckpt, cint, s, nop, any);
    if (st) return st;
    if (nd > 0) WP_CUDA(launch_residual(dsyn, d_obs, L.res, nd, L.partials, residual_parts(nd),
                                        misfit ? misfit : L.misfit, s));
    // Adjoint with the imaging condition of Eq. 2 fused into the stencil.
    WP_CUDA(launch_fill(L.v, (long long)SV * 4 * N, 0.f, s));
    if (M->G.tti) WP_CUDA(launch_fill(L.ef, (long long)2 * SV * N, 0.f, s));
    WP_CUDA(launch_fill(L.img, (long long)S * N, 0.f, s));
    StencilArgs A = base_args(M, g, L);
    set_residual_injection(A, L, g, L.res, nt);
    A.u_in_ss = A.u_out_ss = A.d_in_ss = A.d_out_ss = 4 * N;
    A.img = L.img;
    A.img_ss = N;
    A.h_ss = (long long)hslots * N;
    A.img_scale = inv_dt2;
    // Adjoint steps j = jhi .. jlo (descending), hp(j) the history row of increment j.  On
    // 2-D isotropic grids steps (j, j-1) run as one two-step launch that adds both steps'
    // imaging terms (stencil2.cu), otherwise one step per launch.  v lives in one of two
    // buffers (L.v + {0, 1} N per shot) and its increment in one of two (+ {2, 3} N): a
    // single step updates the increment in place, a pair writes the other buffer.
    const bool two_img = M->G.tz2 > 0 && !M->G.tti;
    const int *roff1 = A.inj_off;
    const InjEntry *rent1 = A.inj;
    const int *roff2 = g->nrec > 0 ? L.t.rec2_off : nullptr;
    const InjEntry *rent2 = g->nrec > 0 ? L.t.rec2_ent : nullptr;
    int cu = 0, cd = 0;
    auto adj_range = [&](int jhi, int jlo, auto hp) -> wp_status {
        for (int j = jhi; j >= jlo;) {
            A.u_in = L.v + (size_t)cu * N;
            A.u_out = L.v + (size_t)(cu ^ 1) * N;
            A.d_in = L.v + (size_t)(2 + cd) * N;
            A.step = j;
            if (two_img && j - 1 >= jlo) {
                A.inj_off = roff2;
                A.inj = rent2;
                A.d_out = L.v + (size_t)(2 + (cd ^ 1)) * N;
                A.u1_out = nullptr;
                A.d1_out = nullptr;
                A.step2 = j - 1;
                A.h2 = hp(j + 1);
                A.h1 = hp(j);
                A.h0 = hp(j - 1);
                WP_CUDA(launch_stencil2(M->G, A, s));
                cd ^= 1;
                j -= 2;
            } else {
                A.inj_off = roff1;
                A.inj = rent1;
                A.d_out = L.v + (size_t)(2 + cd) * N;   // in place
                A.h1 = hp(j + 1);
                A.h0 = hp(j);
                wp_status e = launch_step(M, g, L, A, true, true, s);
                if (e) return e;
                j -= 1;
            }
            cu ^= 1;
        }
        return WP_OK;
    };
    if (full) {
        if ((st = adj_range(nt - 1, 0, [&](int j) { return L.hist + (size_t)j * N; }))) return st;
    } else {
        const int ncp = (nt + cint - 1) / cint;
        StencilArgs F = base_args(M, g, L);
        set_source_injection(F, L, g, wavelet);
        const bool wd = !M->G.tti;   // the forward's (w, d) form, as in forward_sweep
        if (wd) {
            F.wd = 1;
            F.u_in_ss = F.u_out_ss = F.u1_ss = (long long)hslots * N;
            F.d_in_ss = F.d_out_ss = 3 * N;
        } else {
            F.u_in_ss = F.u_out_ss = 3 * N;
            F.d_in_ss = F.d_out_ss = F.d1_ss = (long long)hslots * N;
        }
        const int *off1 = F.inj_off;
        const InjEntry *ent1 = F.inj;
        const int *off2 = g->nsrc > 0 ? L.t.src2_off : nullptr;
        const InjEntry *ent2 = g->nsrc > 0 ? L.t.src2_ent : nullptr;
        const bool two_ok = M->G.tz2 > 0 && !M->G.tti;
        for (int k = ncp - 1; k >= 0; k--) {
            const int n0 = k * cint, n1 = std::min(nt, n0 + cint);
            const float *cp = L.ckpt + (size_t)k * 2 * N;
            const size_t cpitch = (size_t)ncp * 2 * N * sizeof(float);
            WP_CUDA(cudaMemcpy2DAsync(L.u, 3 * N * sizeof(float), cp, cpitch, N * sizeof(float), SV,
                                      cudaMemcpyDeviceToDevice, s));
            WP_CUDA(cudaMemcpy2DAsync(L.hist, (size_t)hslots * N * sizeof(float), cp + N, cpitch,
                                      N * sizeof(float), SV, cudaMemcpyDeviceToDevice, s));
            int it = 0;   // launches of this segment: the u (TTI) or w buffers alternate
            for (int n = n0; n < n1; it++) {
                float *h_n = L.hist + (size_t)(n - n0) * N;
                float *h_n1 = L.hist + (size_t)(n - n0 + 1) * N;
                float *h_n2 = L.hist + (size_t)(n - n0 + 2) * N;
                float *b_in = L.u + (size_t)(it & 1) * N, *b_out = L.u + (size_t)((it + 1) & 1) * N;
                if (wd) {
                    F.u_in = h_n;      // d^n
                    F.d_in = b_in;     // w^{n-1}
                    F.d_out = b_out;
                } else {
                    F.u_in = b_in;
                    F.u_out = b_out;
                    F.d_in = h_n;
                }
                F.step = n;
                if (two_ok && n + 1 < n1) {
                    F.inj_off = off2;
                    F.inj = ent2;
                    if (wd) {
                        F.u1_out = h_n1;
                        F.d1_out = nullptr;
                        F.u_out = h_n2;
                    } else {
                        F.d1_out = h_n1;
                        F.d_out = h_n2;
                    }
                    F.step2 = n + 1;
                    WP_CUDA(launch_stencil2(M->G, F, s));
                    n += 2;
                } else {
                    F.inj_off = off1;
                    F.inj = ent1;
                    if (wd) F.u_out = h_n1;
                    else F.d_out = h_n1;
                    if ((st = launch_step(M, g, L, F, false, false, s))) return st;
                    n += 1;
                }
            }
            if ((st = adj_range(n1 - 1, n0, [&](int j) { return L.hist + (size_t)(j - n0) * N; }))) return st;
        }
    }
    WP_CUDA(launch_shot_sum(L.img, N, S, M->G, true, grad, s));
    return WP_OK;
}

size_t wp_residual_workspace_bytes(long long n) { return (size_t)residual_parts(n) * sizeof(double) + 256; }

wp_status wp_residual(const float *d_syn, const float *d_obs, float *res, long long n,
                      double *misfit, void *ws, size_t ws_bytes, wp_stream stream)
{
    if (n < 0 || !d_syn || !d_obs) return fail(WP_ERR_INVALID, "d_syn and d_obs are required");
    if (n == 0) return WP_OK;
    if (misfit && (!ws || ws_bytes < wp_residual_workspace_bytes(n)))
        return fail(WP_ERR_OOM, "workspace too small for the misfit reduction");
    WP_CUDA(launch_residual(d_syn, d_obs, res, n, (double *)ws, residual_parts(n), misfit,
                            (cudaStream_t)stream));
    return WP_OK;
}

size_t wp_probe_accumulate_workspace_bytes(int nshots, int nt, int r)
{
    if (nshots < 1 || nt < 1 || r < 1 || r > 512) return 0;
    const size_t q = (size_t)nshots * r_pad_of(r) * nt_pad_of(nt) * sizeof(__nv_bfloat16);
    return 256 * 3 + 2 * q + 64 * sizeof(int);
}

wp_status wp_probe_accumulate(const float *A, int cnt, long long npoints, int nshots, const float *Q,
                              int nt, int t0, int r, float scale, float *Pout, void *ws,
                              size_t ws_bytes, wp_stream stream)
{
    float *P = Pout;
    if (!A || !Q || !P || !ws) return fail(WP_ERR_INVALID, "A, Q, P and ws are required");
    if (cnt < 1 || npoints < 1 || nshots < 1 || r < 1 || r > 512 || nt < 1 || t0 < 0 ||
        t0 + cnt > nt || t0 % 8)
        return fail(WP_ERR_INVALID, "need 1 <= r <= 512, 0 <= t0, t0 % 8 == 0, t0 + cnt <= nt");
    if (!aligned16(A) || !aligned16(Q) || !aligned16(P) || !aligned16(ws))
        return fail(WP_ERR_INVALID, "device pointers must be 16-byte aligned");
    if (ws_bytes < wp_probe_accumulate_workspace_bytes(nshots, nt, r))
        return fail(WP_ERR_OOM, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    Carve c(ws);
    int *err = c.take<int>(64);
    const int rp = r_pad_of(r), ntp = nt_pad_of(nt);
    __nv_bfloat16 *qhi = c.take<__nv_bfloat16>((size_t)nshots * rp * ntp);
    __nv_bfloat16 *qlo = c.take<__nv_bfloat16>((size_t)nshots * rp * ntp);
    WP_CUDA(cudaMemsetAsync(err, 0, 64 * sizeof(int), s));
    if (npoints % 128 == 0) {
        // Rows of A are 512-byte aligned: use the pipelined bulk-copy kernel.
        WP_CUDA(launch_probe_images(Q, nshots, nt, r, rp, t0, cnt, 1, qhi, qlo, err + 32, s));
        PipeArgs P{};
            P.ring = A;
        P.ring_ss = (long long)cnt * npoints;
        P.sstride = npoints;
        P.nslots = cnt;
        P.N = npoints;
        P.Np = npoints;
        P.NX = (int)npoints;
        P.NXp = (int)npoints;
        P.ntiles = (int)(npoints / 128);
        P.cnt = cnt;
        P.slot0 = 0;
        P.mode = 0;
        P.img_hi = qhi;
        P.img_lo = qlo;
        P.qlo_nz = err + 32;
        P.nblocks = 1;
        P.ncb = ncb_of(cnt);
        P.blk = 0;
        P.img_div = 1;
        P.r = r;
        P.r_pad = rp;
        P.img_ld = (long long)rp * 64;
        P.P = Pout;
        P.P_pitch = npoints;
        P.P_ss = (long long)r * npoints;
        P.scale = scale;
        P.err = err;
        WP_CUDA(launch_probe_pipe(P, nshots, s));
        return WP_OK;
    }
    WP_CUDA(launch_probe_split(Q, nshots, nt, r, rp, ntp, qhi, qlo, s));
    // this kernel keeps at most 256 probes in tensor memory: one launch per slice of 256
    for (int i0 = 0; i0 < r; i0 += 256) {
        GemmArgs G{};
        G.ring = A;
        G.ring_ss = (long long)cnt * npoints;
        G.nslots = cnt;
        G.N = npoints;
        G.t0 = t0;
        G.cnt = cnt;
        G.slot0 = 0;
        G.mode = 0;
        G.qhi = qhi + (long long)i0 * ntp;
        G.qlo = qlo + (long long)i0 * ntp;
        G.q_ss = (long long)rp * ntp;
        G.nt_pad = ntp;
        G.r = std::min(256, r - i0);
        G.r_pad = std::min(256, rp - i0);
        G.P = P + (long long)i0 * npoints;
        G.P_ss = (long long)r * npoints;
        G.scale = scale;
        G.err = err;
        WP_CUDA(launch_probe_gemm(G, nshots, s));
    }
    return WP_OK;
}

// Range finder (Sec. 2.1): workspace carving shared by the size query and the call.
struct RfLayout {
    int *err;
    __nv_bfloat16 *qhi, *qlo;   // split probe operand of one contraction
    float *Y, *T, *Tt, *Dt, *Yt;
    double *W;
    size_t total;
};

RfLayout rf_layout(int nt, int ncols, int nshots, int d_shared, int r, void *ws)
{
    RfLayout L;
    Carve c(ws);
    const int rp = r_pad_of(r);
    const size_t q = (size_t)nshots * rp * std::max(nt_pad_of(nt), nt_pad_of(ncols));
    const size_t S = (size_t)nshots, nd = d_shared ? 1 : S;
    L.err = c.take<int>(64);
    L.qhi = c.take<__nv_bfloat16>(q);
    L.qlo = c.take<__nv_bfloat16>(q);
    L.Y = c.take<float>(S * nt * r);
    L.T = c.take<float>(S * r * ncols);
    L.Tt = c.take<float>(S * ncols * r);
    L.Dt = c.take<float>(nd * ncols * nt);
    L.Yt = c.take<float>(S * r * nt);
    L.W = c.take<double>(S * r * nt);
    L.total = c.off + 256;
    return L;
}

size_t wp_range_finder_workspace_bytes(int nt, int ncols, int nshots, int d_shared, int r)
{
    if (nt < 1 || ncols < 1 || nshots < 1 || r < 1 || r > 256 || r > nt) return 0;
    return rf_layout(nt, ncols, nshots, d_shared, r, nullptr).total;
}

wp_status wp_range_finder(const float *D, int nt, int ncols, int nshots, int d_shared, int power,
                          const float *Z, int r, float *Q, void *ws, size_t ws_bytes, wp_stream stream)
{
    if (!D || !Z || !Q || !ws) return fail(WP_ERR_INVALID, "D, Z, Q and ws are required");
    if (nt < 1 || ncols < 1 || nshots < 1 || r < 1 || r > 256 || r > nt || power < 1 || power > 8)
        return fail(WP_ERR_INVALID, "need nt, ncols, nshots >= 1, 1 <= r <= min(256, nt), 1 <= power <= 8");
    if (!aligned16(D) || !aligned16(Z) || !aligned16(Q) || !aligned16(ws))
        return fail(WP_ERR_INVALID, "device pointers must be 16-byte aligned");
    const RfLayout L = rf_layout(nt, ncols, nshots, d_shared, r, ws);
    if (ws_bytes < L.total) return fail(WP_ERR_OOM, "workspace %zu < %zu bytes", ws_bytes, L.total);
    cudaStream_t s = (cudaStream_t)stream;
    const int rp = r_pad_of(r);
    const long long dss = d_shared ? 0 : (long long)nt * ncols;
    WP_CUDA(cudaMemsetAsync(L.err, 0, 64 * sizeof(int), s));
    WP_CUDA(cudaMemcpyAsync(L.Y, Z, (size_t)nshots * nt * r * sizeof(float), cudaMemcpyDeviceToDevice, s));
    WP_CUDA(launch_transpose(D, dss, nt, ncols, d_shared ? 1 : nshots, L.Dt, dss, s));
    GemmArgs G{};
    G.t0 = 0;
    G.slot0 = 0;
    G.mode = 0;
    G.qhi = L.qhi;
    G.qlo = L.qlo;
    G.r = r;
    G.r_pad = rp;
    G.scale = 1.f;
    G.err = L.err;
    for (int k = 0; k < power; k++) {
        // T = D^T Y: rows t of D are the contraction's steps, its columns the points
        WP_CUDA(cudaMemsetAsync(L.T, 0, (size_t)nshots * r * ncols * sizeof(float), s));
        WP_CUDA(launch_probe_split(L.Y, nshots, nt, r, rp, nt_pad_of(nt), L.qhi, L.qlo, s));
        G.ring = D;
        G.ring_ss = dss;
        G.nslots = nt;
        G.N = ncols;
        G.cnt = nt;
        G.q_ss = (long long)rp * nt_pad_of(nt);
        G.nt_pad = nt_pad_of(nt);
        G.P = L.T;
        G.P_ss = (long long)r * ncols;
        WP_CUDA(launch_probe_gemm(G, nshots, s));
        // Y = D T, as Y^T = contraction of D^T (rows c) with T^T
        WP_CUDA(launch_transpose(L.T, (long long)r * ncols, r, ncols, nshots, L.Tt, (long long)ncols * r, s));
        WP_CUDA(cudaMemsetAsync(L.Yt, 0, (size_t)nshots * r * nt * sizeof(float), s));
        WP_CUDA(launch_probe_split(L.Tt, nshots, ncols, r, rp, nt_pad_of(ncols), L.qhi, L.qlo, s));
        G.ring = L.Dt;
        G.ring_ss = dss;
        G.nslots = ncols;
        G.N = nt;
        G.cnt = ncols;
        G.q_ss = (long long)rp * nt_pad_of(ncols);
        G.nt_pad = nt_pad_of(ncols);
        G.P = L.Yt;
        G.P_ss = (long long)r * nt;
        WP_CUDA(launch_probe_gemm(G, nshots, s));
        WP_CUDA(launch_cgs2_qr(L.Yt, nt, r, nshots, L.W, k + 1 == power ? Q : L.Y, L.err, s));
    }
    return WP_OK;
}

wp_status wp_offset_image(const wp_model_t *Min, const float *P_u, const float *P_v, int r,
                          int nshots, float scale, int nh, float *out, wp_stream stream)
{
    if (!Min) return fail(WP_ERR_INVALID, "model is NULL");
    if (!P_u || !P_v || !out) return fail(WP_ERR_INVALID, "P_u, P_v and out are required");
    if (r < 1 || r > 512 || nshots < 1 || nh < 0 || nh > 64)
        return fail(WP_ERR_INVALID, "need 1 <= r <= 512, nshots >= 1, 0 <= nh <= 64");
    const GridDev &G = Min->G;
    const bool aligned = Min->probe_layout == WP_PROBES_ALIGNED;
    if (aligned && (!aligned16(P_u) || !aligned16(P_v)))
        return fail(WP_ERR_INVALID, "P_u and P_v must be 16-byte aligned in the aligned layout");
    WP_CUDA(launch_offset_image(P_u, P_v, aligned, G.NX, G.NXp, G.N, aligned ? ring_stride_of(G.Np) : G.N, r,
                                nshots, scale, nh, out, (cudaStream_t)stream));
    return WP_OK;
}

wp_status wp_offset_status(wp_stream stream, double timeout_s)
{
    int *err = nullptr;
    WP_CUDA(offset_err_ptr(&err));
    const wp_status st = wp_stream_status(nullptr, stream, timeout_s);
    if (st != WP_OK) return st;
    int flag = 0;
    WP_CUDA(cudaMemcpy(&flag, err, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) return fail(WP_ERR_TIMEOUT, "a device wait of wp_offset_image gave up");
    return WP_OK;
}

void wp_profile_enable(int on, int capacity) { prof_enable(on, capacity); }

int wp_profile_read(int cls, double *total_ms, long long *count)
{
    return prof_read(cls, total_ms, count);
}

/* Poll a stream with a host-side deadline (never spinning on the device) and report the
 * device error flag kept at the start of every workspace. */
wp_status wp_check_bounded_wait(void *ws, size_t ws_bytes, wp_stream stream)
{
    if (!ws || ws_bytes < 256 || !aligned16(ws)) return fail(WP_ERR_INVALID, "need a 16-byte aligned workspace of >= 256 bytes");
    cudaStream_t s = (cudaStream_t)stream;
    WP_CUDA(cudaMemsetAsync(ws, 0, 64 * sizeof(int), s));
    WP_CUDA(launch_bounded_wait((int *)ws, s));
    return WP_OK;
}

wp_status wp_stream_status(const void *ws, wp_stream stream, double timeout_s)
{
    cudaStream_t s = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(s);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return fail(WP_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(WP_ERR_TIMEOUT, "stream did not finish within %.3f s", timeout_s);
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    if (!ws) return WP_OK;
    int flag = 0;
    WP_CUDA(cudaMemcpy(&flag, ws, sizeof flag, cudaMemcpyDeviceToHost));
    if (flag) return fail(WP_ERR_TIMEOUT, "a device wait gave up (error flag %d)", flag);
    return WP_OK;
}

}  // extern "C"
