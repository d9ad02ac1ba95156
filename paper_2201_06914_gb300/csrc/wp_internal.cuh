// Internal declarations shared by the CUDA translation units of libwp.so.
// Nothing here is part of the C ABI (include/wp.h).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/wp.h"

namespace wp {

// ---------------------------------------------------------------------------------------
// Padded grid + absorbing layer, as the kernels see it.
// ---------------------------------------------------------------------------------------
struct GridDev {
    int ndim;
    int NX, NY, NZ;        // padded sizes (NY = 1 in 2-D)
    int NXp;               // row pitch of internal fields: NX rounded up to 4 floats
    long long Np;          // points of an internal field: NXp * NY * NZ
    int nx, ny, nz, nbl;   // interior sizes, absorbing width
    float ihx2, ihy2, ihz2; // 1/h^2 per axis
    float lrz, lry, lapK;   // hx^2/hz^2, hx^2/hy^2 (0 in 2-D), 2 (1 + lrz + lry)
    // sigma0 * dt / 2 per axis: sigma*dt/2 = sum_axes hs0 * (d/nbl)^2
    float hs0x, hs0y, hs0z;
    float inv_nbl;
    long long N;
    int tx;                // columns of one stencil tile along x (a multiple of 4)
    int tz;                // planes marched by one block (>= 1)
    int tz2;               // planes per two-step segment (0: two-step launches off)
    float hx, hy, hz;      // grid spacing (m)
    int tti;               // 1: pseudo-acoustic TTI (two fields per shot)
};

// 8th-order central second-derivative weights (Fornberg): offsets 1..4 (the centre weight
// is minus twice their sum, which the difference form below uses implicitly).
#define WP_C1 (8.0f / 5.0f)
#define WP_C2 (-1.0f / 5.0f)
#define WP_C3 (8.0f / 315.0f)
#define WP_C4 (-1.0f / 560.0f)

// sigma*dt/2 at one padded index of one axis.
__device__ __forceinline__ float damp_term(int i, int n, int nbl, float hs0, float inv_nbl)
{
    int d = 0;
    if (i < nbl) d = nbl - i;
    else if (i >= nbl + n) d = i - (nbl + n - 1);
    float f = (float)d * inv_nbl;
    return hs0 * f * f;
}

__device__ __forceinline__ float damp_at(const GridDev &G, int x, int y, int z)
{
    float s = damp_term(x, G.nx, G.nbl, G.hs0x, G.inv_nbl) +
              damp_term(z, G.nz, G.nbl, G.hs0z, G.inv_nbl);
    if (G.ndim == 3) s += damp_term(y, G.ny, G.nbl, G.hs0y, G.inv_nbl);
    return s;
}

// ---------------------------------------------------------------------------------------
// Injection table: entries grouped by (shot, stencil tile, plane) in CSR form;
// a = local x + TX * local y, b = global z.
// ---------------------------------------------------------------------------------------
struct InjEntry {
    int a;
    int b;
    int trace;
    float w;
};

// Stencil tiling (the host builds injection tables with the same tiling).  A block owns a
// TX x TY patch of (x, y) columns and marches `tz` planes along z (TX and tz are chosen by
// the host and stored in GridDev::tx and GridDev::tz).
// Each thread owns 4 adjacent columns (one float4), so a tile is (4 * threads_x) x TY.
//   2-D: TY = 1, TX = 128 (32 threads) or 256 (64 threads), whichever pads NX less;
//   3-D: 16 x 8 threads, 64 x 8 columns.
constexpr int T2Y = 1;
constexpr int T3TX = 16, T3X = 4 * T3TX, T3Y = 8;
constexpr int RAD = 4;                               // stencil radius (space order 8)

struct StencilArgs {
    const float *u_in;  long long u_in_ss;   // u^n (or v^{j+1}), shot stride
    const float *d_in;  long long d_in_ss;   // increment u^n - u^{n-1}
    float *u_out;       long long u_out_ss;  // u^{n+1}
    float *d_out;       long long d_out_ss;  // increment u^{n+1} - u^n (may alias d_in)
    const float *b;                          // dt^2 / m, N values shared by the shots
    // injection of  w * sign * traces[shot*tr_ss + step*tr_ts + trace*tr_rs]
    const int *inj_off; const InjEntry *inj;
    const float *traces; long long tr_ss, tr_ts, tr_rs; int step; float tr_sign;
    // recording: out[shot*g_ss + g_row*nrec + rec] = sum_c w[c] * u_in[idx[c]]
    const int *g_idx; const float *g_w; int nrec; int ncorner;
    float *g_out; long long g_ss; int g_row; int do_gather;
    // exact imaging: img[p] += img_scale * (cp*h1[p] - cm*h0[p]) * u_out[p]; a two-step
    // launch adds both steps: (cp*h2 - cm*h1) * u1 + (cp*h1 - cm*h0) * u_out, u1 the first
    // step's output
    float *img; long long img_ss;
    const float *h2; const float *h1; const float *h0; long long h_ss; float img_scale;
    int nshots;
    int *err;          // device error flag (a bounded wait gave up)
    // two-step launches (stencil2.cu): step-1 fields (NULL: kept on chip), trace row of step 2
    float *u1_out; long long u1_ss;
    float *d1_out; long long d1_ss;
    int step2;
    // pending recording row of a preceding two-step launch:
    //   out[shot*g_ss + gp_row*nrec + rec] = sum_c w[c] * (gp_u[idx[c]] + gp_d[idx[c]])
    const float *gp_u; long long gp_u_ss;
    const float *gp_d; long long gp_d_ss;
    int gp_row; int do_pend;
    // (w, d) form (forward, isotropic): X = d (stencil field, u_in/u_out), Y = w = L u
    // (d_in/d_out).  u is never formed, so recording keeps u at the receiver corners in
    // g_acc[shot][rec][corner] (FP64), adding the increment of each recorded step.
    int wd;
    double *g_acc;
};

// Recording blocks shared by the stencil launches: block gb of the row read from u_in
// (do_gather) and then of the pending row (do_pend), one receiver per thread.
__device__ __forceinline__ void gather_block(const StencilArgs &A, int gblock)
{
    const int shot = blockIdx.y;
    const int rec = gblock * blockDim.x + threadIdx.x;
    if (rec >= A.nrec) return;
    const float *u = A.u_in + (long long)shot * A.u_in_ss;
    const long long base = ((long long)shot * A.nrec + rec) * A.ncorner;
    float acc = 0.f;
    for (int c = 0; c < A.ncorner; c++) acc += A.g_w[base + c] * u[A.g_idx[base + c]];
    A.g_out[(long long)shot * A.g_ss + (long long)A.g_row * A.nrec + rec] = acc;
}

__device__ __forceinline__ void gather_pend(const StencilArgs &A, int gblock)
{
    const int shot = blockIdx.y;
    const int rec = gblock * blockDim.x + threadIdx.x;
    if (rec >= A.nrec) return;
    const float *u = A.gp_u + (long long)shot * A.gp_u_ss;
    const float *d = A.gp_d + (long long)shot * A.gp_d_ss;
    const long long base = ((long long)shot * A.nrec + rec) * A.ncorner;
    float acc = 0.f;
    for (int c = 0; c < A.ncorner; c++) {
        const int i = A.g_idx[base + c];
        acc += A.g_w[base + c] * (u[i] + d[i]);   // u^{n+1} = u^n + d^{n+1}, as the step adds it
    }
    A.g_out[(long long)shot * A.g_ss + (long long)A.gp_row * A.nrec + rec] = acc;
}

// (w, d) form: u at the receiver corners is kept in g_acc and advanced by the increments
// in step order: first d^{n} of the pending row (the first step of a preceding two-step
// launch, stored at gp_d), then d of the input (u_in = d^n of this launch), each followed by
// its record row.  One thread owns one receiver; corners shared by two receivers are kept
// in both slots, with the same additions.
__device__ __forceinline__ void gather_wd(const StencilArgs &A, int gblock)
{
    const int shot = blockIdx.y;
    const int rec = gblock * blockDim.x + threadIdx.x;
    if (rec >= A.nrec) return;
    const long long base = ((long long)shot * A.nrec + rec) * A.ncorner;
    double *acc = A.g_acc + base;
    float *out = A.g_out + (long long)shot * A.g_ss;
    if (A.do_pend) {
        const float *d = A.gp_d + (long long)shot * A.gp_d_ss;
        double s = 0.0;
        for (int c = 0; c < A.ncorner; c++) {
            const double v = acc[c] + (double)d[A.g_idx[base + c]];
            acc[c] = v;
            s += (double)A.g_w[base + c] * v;
        }
        out[(long long)A.gp_row * A.nrec + rec] = (float)s;
    }
    if (A.do_gather) {
        const float *d = A.u_in + (long long)shot * A.u_in_ss;
        double s = 0.0;
        for (int c = 0; c < A.ncorner; c++) {
            const double v = acc[c] + (double)d[A.g_idx[base + c]];
            acc[c] = v;
            s += (double)A.g_w[base + c] * v;
        }
        out[(long long)A.g_row * A.nrec + rec] = (float)s;
    }
}

// Recording blocks a launch needs per shot (blocks of `nt` threads).
__host__ __device__ inline int gather_blocks(const StencilArgs &A, int nt)
{
    const int ng = (A.nrec + nt - 1) / nt;
    if (A.wd) return (A.do_gather || A.do_pend) ? ng : 0;
    return ng * ((A.do_gather ? 1 : 0) + (A.do_pend ? 1 : 0));
}

__device__ __forceinline__ void gather_rows(const StencilArgs &A, int gb)
{
    if (A.wd) {
        gather_wd(A, gb);
        return;
    }
    const int ng = (A.nrec + blockDim.x - 1) / blockDim.x;
    if (A.do_gather) {
        if (gb < ng) {
            gather_block(A, gb);
            return;
        }
        gb -= ng;
    }
    if (A.do_pend && gb < ng) gather_pend(A, gb);
}

// TTI step: fields of shot s are the virtual shots 2s (p) and 2s+1 (q); strides below are
// per virtual shot.
struct TtiArgs {
    const float *u_in; long long u_in_ss;
    const float *d_in; long long d_in_ss;
    float *u_out; long long u_out_ss;
    float *d_out; long long d_out_ss;
    const float *b;                                    // dt^2/m (padded)
    const float *E, *Sd, *ax, *ay, *az;                // padded parameter fields
    float *t; long long t_ss;                          // scratch Dr x per virtual shot
    int adjoint;
    // adjoint: e = E a + S b (virtual shot 2s) and f = S a + b (2s+1) of the input fields,
    // and the same combinations of the updated fields written by this step
    const float *ef_in; float *ef_out; long long ef_ss;
    float *img; long long img_ss;                      // exact imaging (per real shot) or NULL
    const float *h1, *h0; long long h_ss; float img_scale;
    int nshots;                                        // real shots
    int *err;                                          // device error flag (a bounded wait gave up)
};

// Point-list injection after a TTI update: value = sign * w * traces[s*tr_ss + step*tr_ts
// + j*tr_rs] at corner `idx` of point j of shot s; both fields (forward) or the first.
struct TtiInject {
    const int *idx; const float *w; int npts, ncorner;
    const float *traces; long long tr_ss, tr_ts, tr_rs; int step; float sign; int both;
};

// Tile counts of a grid in the stencil tiling.
inline int tile_x(const GridDev &G) { return G.tx; }
inline int tile_y(const GridDev &G) { return G.ndim == 2 ? T2Y : T3Y; }
inline int tiles_x(const GridDev &G) { return (G.NX + tile_x(G) - 1) / tile_x(G); }
inline int tiles_y(const GridDev &G) { return (G.NY + tile_y(G) - 1) / tile_y(G); }
inline int tiles_z(const GridDev &G) { return (G.NZ + G.tz - 1) / G.tz; }
inline int stencil_tiles(const GridDev &G) { return tiles_x(G) * tiles_y(G) * tiles_z(G); }
// Injection-table keys: one per (tile, plane within the tile).
inline long long stencil_keys(const GridDev &G) { return (long long)stencil_tiles(G) * G.tz; }
// Two-step tiling (2-D, stencil2.cu): tiles of G.tx columns starting at t*(tx - 8) - 4
// (neighbours overlap by 8 columns), segments of G.tz2 planes extended by 4 on each side.
inline int core2_x(const GridDev &G) { return G.tx - 2 * RAD; }
inline int tiles2_x(const GridDev &G) { return (G.NXp + core2_x(G) - 1) / core2_x(G); }
inline int tiles2_z(const GridDev &G) { return (G.NZ + G.tz2 - 1) / G.tz2; }
inline int stencil2_tiles(const GridDev &G) { return tiles2_x(G) * tiles2_z(G); }
inline long long stencil2_keys(const GridDev &G) { return (long long)stencil2_tiles(G) * (G.tz2 + 2 * RAD); }

// Probe contraction arguments.
struct GemmArgs {
    const float *ring; long long ring_ss; int nslots; long long N;
    int t0, cnt;     // absolute first time index of the block (probe row), valid steps
    int slot0;       // ring slot holding step t0 (forward: increment t0)
    int mode;        // 0: A_t = ring[slot(t)]; 1: A_t = cp*ring[slot(t+1)] - cm*ring[slot(t)]
    const __nv_bfloat16 *qhi, *qlo; long long q_ss; int nt_pad; // [shot][r_pad][nt_pad]
    int r, r_pad;
    float *P; long long P_ss;   // [shot][r][N] accumulated in place
    float scale;
    // fused imaging after the last block: img[p] = img_scale * sum_i Pu[i][p] * P[i][p]
    const float *Pu; long long Pu_ss; float *img; long long img_ss; float img_scale; int do_img;
    GridDev G;
    int *err;
};

// Pipelined probe contraction over the time-step ring (probe_pipe.cu).  The ring slot
// stride is a multiple of 128 floats so that every 128-point row segment can be fetched
// with one 512-byte bulk copy.
struct PipeArgs {
    const float *ring; long long ring_ss; long long sstride; int nslots;
    long long N;            // points per shot in the dense layout of P (unpadded)
    long long Np;           // points per ring row (padded layout, pitch NXp)
    int NX, NXp;            // row length and row pitch: ring point p -> user point
    int ntiles;             // ceil(Np / 128)
    int cnt, slot0, mode;   // steps in the block, ring slot of its first step, A mode
    const __nv_bfloat16 *img_hi, *img_lo;  // swizzled probe images, see launch_probe_images
    long long img_ld;       // elements from one probe image to the next (r_pad * 64)
    int nblocks, ncb, blk;  // images per shot = nblocks * ncb; this block's index
    int img_div;            // virtual shots per probe-image shot (2 for TTI fields)
    int r, r_pad;
    float *P; long long P_ss; long long P_pitch; float scale;   // P rows P_pitch floats apart
    const int *qlo_nz;      // device flag set by launch_probe_images when a probe value is not
                            // exactly a bfloat16 (nullptr: assume so): without it the products
                            // with the probes' lo part (all zero, e.g. Rademacher +-1) are skipped
    int p_zero;             // 1: P holds no earlier blocks (first block): write, do not read
    GridDev G;
    int *err;
};

// ---------------------------------------------------------------------------------------
// Launchers (host), defined in the .cu files.
// ---------------------------------------------------------------------------------------
cudaError_t launch_stencil(const GridDev &G, const StencilArgs &A, bool imaging, cudaStream_t s);
// Tile width for a grid (host only), and the stencil blocks one SM holds for that tiling.
int stencil_choose_tx(const GridDev &G);
int stencil_blocks_per_sm(const GridDev &G);
// Two time steps per launch (2-D isotropic; G.tz2 >= 1).
cudaError_t launch_stencil2(const GridDev &G, const StencilArgs &A, cudaStream_t s);
int stencil2_blocks_per_sm(const GridDev &G);
int device_sm_count();
cudaError_t launch_gather(const GridDev &G, const StencilArgs &A, cudaStream_t s);
cudaError_t launch_probe_gemm(const GemmArgs &A, int nshots, cudaStream_t s);
cudaError_t launch_probe_split(const float *Q, int nshots, int nt, int r, int r_pad, int nt_pad,
                               __nv_bfloat16 *qhi, __nv_bfloat16 *qlo, cudaStream_t s);
cudaError_t launch_probe_pipe(const PipeArgs &A, int nshots, cudaStream_t s);
typedef CUresult (*encode_tiled_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
// cuTensorMapEncodeTiled through the runtime's driver entry point (nullptr if unavailable).
encode_tiled_fn encoder();
// out[h + nh][p] = scale * sum_s sum_i Pu[s][i][p + h] * Pv[s][i][p - h] along x (Eq. 4).
// Dense operands: rows of N points (x pitch NX); aligned: rows of `pitch` floats with the
// points at x pitch NXp.  out is dense, (2 nh + 1) x N.
cudaError_t launch_offset_image(const float *Pu, const float *Pv, bool aligned, int NX, int NXp, long long N,
                                long long pitch, int r, int nshots, float scale, int nh, float *out,
                                cudaStream_t s);
// Device address of the offset kernels' error flag (static device memory).
cudaError_t offset_err_ptr(int **p);
// g[u] = scale * sum_s sum_i Pu[s][i][.] * Pv[s][i][w(u)]: Pv in the row-aligned layout
// (rows of `pitch` floats, point u at w(u) = row * NXp + x), Pu dense (rows of N, at u) or,
// with pu_aligned, in the same layout as Pv
cudaError_t launch_probe_dot(const float *Pu, bool pu_aligned, const float *Pv, long long N, int NX, int NXp,
                             long long pitch, int r, int nshots, float scale, float *g, cudaStream_t s);
// row-aligned probe rows -> dense layout
cudaError_t launch_p_to_user(const float *in, long long pitch, long long rows, long long N, int NX,
                             int NXp, float *out, cudaStream_t s);
cudaError_t launch_tti_params(const GridDev &G, const float *eps, const float *delta,
                              const float *theta, const float *phi, float *E, float *Sd,
                              float *ax, float *ay, float *az, cudaStream_t s);
cudaError_t launch_tti_step(const GridDev &G, const TtiArgs &T, const TtiInject &J, cudaStream_t s);
cudaError_t launch_maxval(const float *x, long long n, float *out, cudaStream_t s);
// *count += #{i : !(a[i] <= b[i]) or a value not finite} (count zeroed by the caller)
cudaError_t launch_count_greater(const float *a, const float *b, long long n, int *count, cudaStream_t s);
// A single bounded device wait that nothing completes: sets *err after about one second.
cudaError_t launch_bounded_wait(int *err, cudaStream_t s);
// Probe images: for block b (first step t_first + b*Tb) and 64-step chunk c, an r_pad x 64
// bf16 tile in the 128-byte-swizzled K-major layout of tcgen05 (hi and lo parts).
// lo_nz (device int, zeroed by the caller) becomes 1 if any probe value has a nonzero lo part.
cudaError_t launch_probe_images(const float *Q, int nshots, int nt, int r, int r_pad,
                                int t_first, int Tb, int nblocks, __nv_bfloat16 *hi,
                                __nv_bfloat16 *lo, int *lo_nz, cudaStream_t s);
// out[s][c][r] = in[s][r][c] (R x C per matrix, nmat matrices).
cudaError_t launch_transpose(const float *in, long long in_ss, int R, int C, int nmat, float *out,
                             long long out_ss, cudaStream_t s);
// Thin QR (CGS2, FP64) of Yt[s][i][t] (nt x r, column-major per shot) -> Q[s][t][i].
cudaError_t launch_cgs2_qr(const float *Yt, int nt, int r, int nshots, double *W, float *Q, int *err,
                           cudaStream_t s);
cudaError_t launch_b_field(const float *m, double dt2, const GridDev &G, float *b, cudaStream_t s);
cudaError_t launch_fill(float *p, long long n, float v, cudaStream_t s);
// g[p] = sum_s img[s][.] for the N user-layout points; `padded` images use pitch G.NXp.
cudaError_t launch_shot_sum(const float *img, long long img_ss, int nshots, const GridDev &G,
                            bool padded, float *g, cudaStream_t s);
cudaError_t launch_minmax(const float *m, long long N, float *out2, int *bad, cudaStream_t s);
cudaError_t launch_residual(const float *a, const float *b, float *res, long long n,
                            double *partials, int nparts, double *misfit, cudaStream_t s);
int residual_parts(long long n);

void count_launch(long long k = 1);
// Kernel classes for the optional event timing (wp_profile_*).
enum { PROF_STENCIL = 0, PROF_GEMM = 1, PROF_OTHER = 2, PROF_STENCIL2 = 3, PROF_STENCIL2_IMG = 4, PROF_NCLASS = 5 };
void prof_enable(int on, int capacity);
cudaEvent_t prof_begin(int cls, cudaStream_t s);
void prof_end(int cls, cudaEvent_t began, cudaStream_t s);
int prof_read(int cls, double *total_ms, long long *count);
// Sets the thread-local message returned by wp_last_error().
void set_last_error(const char *msg);
long long launches();
size_t probe_gemm_smem(int r_pad);

// ---------------------------------------------------------------------------------------
// PTX helpers for tcgen05 / mbarrier (sm_100a family).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~2^31 clock cycles (about one second) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > (1ll << 31)) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk asynchronous copy global -> shared (16-byte aligned, size a multiple of 16) that
// signals completion of its bytes on an mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 16-byte asynchronous copy global -> shared; `bytes` = 0 writes zeros (the address is
// still a valid one).
__device__ __forceinline__ void cp_async16(uint32_t dst, const float *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Executed by one full warp.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(ncols)
                 : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, bf16 inputs, fp32 accumulation, issued by one thread.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 32 lanes x 32 bit, 16 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// try_wait that lets the hardware suspend the thread for up to `ns` nanoseconds (it wakes
// as soon as the phase completes), so waiting roles do not spin on the issue slots the
// working warps need.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Bounded, sleeping wait shared by the roles of a pipelined kernel: gives up (and raises
// the block's abort flag) after about 2^31 cycles, or returns at once once another role
// has raised it.
__device__ __forceinline__ bool mbar_wait_abortable(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    const long long t0 = clock64();
    while (!mbar_try_wait_sleep(bar, parity, 100000u)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > (1ll << 31)) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// Named barrier `id` over `count` threads that returns to every one of them whether any
// of them passed failed = true (so a group leaves its loop together).
template <int ID, int COUNT>
__device__ __forceinline__ bool bar_any(bool failed)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred q, p;\n\t"
                 "setp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.or.pred p, %2, %3, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r) : "r"((uint32_t)failed), "n"(ID), "n"(COUNT) : "memory");
    return r != 0;
}

// (a, b) -> bf16 pairs hi = rn(a, b) and lo = rn(a - hi_a, b - hi_b), a in the low halves
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups `sbo`
// bytes apart (1024: packed atoms; tcgen05 descriptor format: start>>4 at [0,14), LBO>>4 at [16,30), SBO>>4 at
// [32,46), version 1 at [46,48), layout type SWIZZLE_128B = 2 at [61,64)).
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr, uint32_t sbo = 1024)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D fp32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

}  // namespace wp
