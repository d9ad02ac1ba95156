// Acoustic time-step kernels (forward and adjoint use the same kernel, Sec. 2.2).
//
// One launch advances every shot of a batch by one leapfrog step of
//   m (u_tt + sigma u_t) - Laplacian(u) = q
// written in increment form to limit FP32 rounding growth: with d^n = u^n - u^{n-1},
//   a^n     = (dt^2/m) (L u^n + q^n)                  (= dt^2 * u_tt^n)
//   d^{n+1} = ((1 - sigma dt/2) d^n + a^n) / (1 + sigma dt/2)
//   u^{n+1} = u^n + d^{n+1}
// which is algebraically the centred scheme (1+sigma dt/2)u^{n+1} - 2u^n +
// (1-sigma dt/2)u^{n-1} = a^n.  L is the 8th-order Laplacian evaluated in difference
// form, sum_k c_k ((u[+k] - u[0]) + (u[-k] - u[0])), with zero values beyond the grid.
//
// Data movement: a block owns a tile of (x, y) columns (2-D: 512 x 1, 3-D: 64 x 8; every
// thread owns 4 adjacent columns as one float4) and marches `tz` planes along z.  Planes
// are staged through shared memory with 16-byte cp.async copies that zero-fill outside the
// grid (the Dirichlet exterior costs nothing): a ring holds the u tiles of planes z-4 .. z+4
// with their x/y halos plus LA planes in flight, a second ring the increment and dt^2/m of
// the plane being updated.  Internal fields use a row pitch NXp (NX rounded up to 4) so
// that every float4 is 16-byte aligned; the padding columns are kept at zero.
//
// Fused into the same launch:
//   - injection of point sources (forward) or of the receiver residual (adjoint): each
//     warp adds the entries of its columns from the (tile, plane) keys of a CSR table in
//     shared memory, so no atomics reach global memory and no block barrier is needed;
//   - recording d = R u^n of the input wavefield (extra blocks after the stencil tiles),
//     and the pending row of a preceding two-step launch (stencil2.cu);
//   - the exact imaging condition of Eq. 2 (template flag IMG): g += u_tt^j * v^j with
//     u_tt^j rebuilt from two stored forward increments.
#include <cstdlib>

#include "stencil_step.cuh"

namespace wp {

using step::P4;


// Block = TXT x TY threads; thread (lx, ly) owns the 4 adjacent columns
// x = x0 + 4*lx + j (j < 4) of row y = y0 + ly, so a tile is TX = 4*TXT columns wide.  The
// block marches planes z0 .. z1-1.
//
// Along z every thread keeps its own float4 of the nine planes z-4 .. z+4 in registers
// (the march loop is unrolled by U planes and the window slides by U once per group).
// Shared memory only serves the neighbours inside a plane: a ring of NU u tiles with x/y
// halos, filled with 16-byte cp.async copies that zero-fill outside the grid (the Dirichlet
// exterior costs nothing), and a ring of NDB tiles holding the increment and dt^2/m of the
// planes being updated.  LA planes are in flight; one barrier per plane.
#ifndef WP_STENCIL_U
#define WP_STENCIL_U 3
#endif
#ifndef WP_STENCIL_LA3D
#define WP_STENCIL_LA3D 3
#endif
// NA: fields staged per plane in the increment ring (2: the increment and dt^2/m; 5 for the
// 2-D exact-imaging variant, which also stages the two history rows and the image it updates,
// so that their loads do not sit in the step's critical path).
template <int TXT, int TY, int NA = 2>
struct StencilShape {
    static constexpr int TX = 4 * TXT;
    static constexpr int HY = TY > 1 ? RAD : 0;
    static constexpr int NT = TXT * TY;
    static constexpr int W = TX + 2 * RAD;
    static constexpr int H = TY + 2 * HY;
    static constexpr int U = WP_STENCIL_U;           // planes per unrolled group
    static constexpr int LA = TY > 1 ? WP_STENCIL_LA3D : 3;   // planes in flight: u z+5.., db z+1..
    static constexpr int NU = 8;                     // u ring: planes z .. z+4+LA
    static constexpr int NDB = 4;                    // increment/model ring
    static constexpr int USLOT = H * W;              // floats
    static constexpr int DBSLOT = NA * TY * TX;      // floats
    static constexpr int UCH = USLOT / 4;            // 16-byte chunks per u tile
    static constexpr int DBCH = DBSLOT / 4;
    static constexpr int UK = (UCH + NT - 1) / NT;   // u chunks per thread
    static constexpr int DK = (DBCH + NT - 1) / NT;  // increment/model chunks per thread
    static constexpr size_t SMEM = (size_t)(NU * USLOT + NDB * DBSLOT) * sizeof(float);
    // resident blocks per SM (launch bound: 2-D registers <= 128; 3-D <= 168, the y
    // neighbours add 32 live registers)
    static constexpr int MINB = TY > 1 ? 3 : 8192 / (NT * 16) > 16 ? 16 : 8192 / (NT * 16);
    static_assert(RAD + 1 + LA <= NU && LA + 1 <= NDB, "rings");
    static_assert((NU & (NU - 1)) == 0 && (NDB & (NDB - 1)) == 0, "ring sizes are powers of two");
};

template <int TXT, int TY, bool IMG>
constexpr int stencil_na() { return (IMG && TY == 1) ? 5 : 2; }

template <int TXT, int TY, bool IMG, bool WD>
__global__ void __launch_bounds__(TXT *TY, StencilShape<TXT, TY, stencil_na<TXT, TY, IMG>()>::MINB)
    stencil_kernel(const GridDev G, const StencilArgs A)
{
    using S = StencilShape<TXT, TY, stencil_na<TXT, TY, IMG>()>;
    constexpr int TX = S::TX, HY = S::HY, W = S::W, NT = S::NT, LA = S::LA, U = S::U;
    constexpr int NU = S::NU, NDB = S::NDB;
    constexpr uint32_t USZ = S::USLOT * 4, DSZ = S::DBSLOT * 4;   // slot bytes
    extern __shared__ float4 smem4[];
    float *uring = (float *)smem4;
    float *dbring = uring + NU * S::USLOT;
    __shared__ float sq[TY][TX];
    __shared__ int inj_lo, inj_hi;

    const int ntx = (G.NX + TX - 1) / TX, nty = (G.NY + TY - 1) / TY;
    const int ntiles = ntx * nty * ((G.NZ + G.tz - 1) / G.tz);
    if ((int)blockIdx.x >= ntiles) {
        gather_rows(A, blockIdx.x - ntiles);
        return;
    }
    const int tid = threadIdx.x, tile = blockIdx.x;
    const long long sh = blockIdx.y;
    const int lx = tid % TXT, ly = tid / TXT;
    const int x0 = (tile % ntx) * TX, y0 = ((tile / ntx) % nty) * TY;
    const int z0 = (tile / (ntx * nty)) * G.tz, z1 = min(z0 + G.tz, G.NZ);
    const int nplanes = z1 - z0;
    const int NXp = G.NXp, PS = G.NXp * G.NY;
    const float *__restrict__ u = A.u_in + sh * A.u_in_ss;

    // Copy descriptors of this thread (fixed across planes): shared-memory byte offset,
    // global address at plane 0 (a valid address even for chunks outside the grid in x/y,
    // which copy 0 bytes and so zero-fill).
    uint32_t us[S::UK];
    const float *ug[S::UK];
    int un16[S::UK];
#pragma unroll
    for (int k = 0; k < S::UK; k++) {
        const int c = tid + k * NT;
        const int r = c / (W / 4), k4 = c % (W / 4);
        const int x = x0 - RAD + 4 * k4, y = y0 - HY + r;
        const bool v = c < S::UCH && x >= 0 && x < NXp && y >= 0 && y < G.NY;
        un16[k] = v ? 16 : 0;
        us[k] = (uint32_t)(r * W + 4 * k4) * 4;
        ug[k] = u + (v ? y * NXp + x : 0);
    }
    uint32_t ds[S::DK];
    const float *dg[S::DK];
    int dn16[S::DK];
#pragma unroll
    for (int k = 0; k < S::DK; k++) {
        const int c = tid + k * NT;
        const int a = c / (TY * TX / 4), rem = c % (TY * TX / 4);
        const int r = rem / (TX / 4), k4 = rem % (TX / 4);
        const int x = x0 + 4 * k4, y = y0 + r;
        const bool v = c < S::DBCH && x < NXp && y < G.NY;
        dn16[k] = v ? 16 : 0;
        ds[k] = (uint32_t)(a * TY * TX + r * TX + 4 * k4) * 4;
        const float *src = a == 0 ? A.d_in + sh * A.d_in_ss
                         : a == 1 ? A.b
                         : a == 2 ? A.h1 + sh * A.h_ss
                         : a == 3 ? A.h0 + sh * A.h_ss
                                  : A.img + sh * A.img_ss;
        dg[k] = src + (v ? y * NXp + x : 0);
    }
    const uint32_t su0 = (uint32_t)__cvta_generic_to_shared(uring);
    const uint32_t sd0 = (uint32_t)__cvta_generic_to_shared(dbring);
    // u plane k (< NZ) into ring slot (k - z0) mod NU; planes beyond the grid are never read
    auto issue_u = [&](int k) {
        if (k >= G.NZ) return;
        const uint32_t base = su0 + (uint32_t)((k - z0) & (NU - 1)) * USZ;
        const long long ko = (long long)k * PS;
#pragma unroll
        for (int q = 0; q < S::UK; q++)
            if ((q + 1) * NT <= S::UCH || tid + q * NT < S::UCH) cp_async16(base + us[q], ug[q] + ko, un16[q]);
    };
    // increment/model plane k (< z1) into ring slot (k - z0) mod NDB
    auto issue_db = [&](int k) {
        if (k >= z1) return;
        const uint32_t base = sd0 + (uint32_t)((k - z0) & (NDB - 1)) * DSZ;
        const long long ko = (long long)k * PS;
#pragma unroll
        for (int q = 0; q < S::DK; q++)
            if ((q + 1) * NT <= S::DBCH || tid + q * NT < S::DBCH) cp_async16(base + ds[q], dg[q] + ko, dn16[q]);
    };

    // Prologue.  Group g < LA holds u plane z0+4+g and db plane z0+g; group 0 also holds
    // the u planes z0 .. z0+3.  Planes z0-4 .. z0-1 are only needed in the window and are
    // read straight from global memory.
#pragma unroll
    for (int k = 0; k < RAD; k++) issue_u(z0 + k);
#pragma unroll
    for (int g = 0; g < LA; g++) {
        issue_u(z0 + RAD + g);
        issue_db(z0 + g);
        cp_async_commit();
    }
    // March indices with injection entries (sources or receivers in this tile).
    const int *off = A.inj ? A.inj_off + sh * ((long long)ntiles * G.tz + 1) : nullptr;
    const long long key0 = (long long)tile * G.tz;
    const bool tile_inj = off && off[key0] < off[key0 + nplanes];
    if (tid == 0) {
        inj_lo = 1 << 30;
        inj_hi = -1;
    }
    __syncthreads();
    if (tile_inj)
        for (int t = tid; t < nplanes; t += NT)
            if (off[key0 + t] < off[key0 + t + 1]) {
                atomicMin(&inj_lo, t);
                atomicMax(&inj_hi, t);
            }

    const float *tr = tile_inj ? A.traces + sh * A.tr_ss + (long long)A.step * A.tr_ts : nullptr;
    const int gy = y0 + ly, xc = x0 + 4 * lx;
    const bool row_ok = gy < G.NY && xc < NXp;   // this thread's float4 lies in the field
    float sdx[4];
#pragma unroll
    for (int j = 0; j < 4; j++)
        sdx[j] = damp_term(xc + j, G.nx, G.nbl, G.hs0x, G.inv_nbl) +
                 (TY > 1 ? damp_term(gy, G.ny, G.nbl, G.hs0y, G.inv_nbl) : 0.f);
    // all four columns outside the x (and y) absorbing layers
    const bool col_int = sdx[0] == 0.f && sdx[1] == 0.f && sdx[2] == 0.f && sdx[3] == 0.f;
    const bool has_pad = xc + 4 > G.NX;          // some of the 4 columns are row padding
    const long long own = (long long)gy * NXp + xc;
    float *uo = A.u_out + sh * A.u_out_ss + own;
    float *dout = A.d_out + sh * A.d_out_ss + own;

    // win[ph + 4 + k] = own four columns of plane zb + ph + k within a group starting at zb
    P4 win[2 * RAD + U];
#pragma unroll
    for (int k = 0; k < RAD; k++) {
        const int zz = z0 - RAD + k;
        win[k] = (row_ok && zz >= 0) ? *(const P4 *)(u + (long long)zz * PS + own) : step::zero();
    }
    const uint32_t ub = su0 + (uint32_t)((ly + HY) * W * 4) + (uint32_t)(RAD + 4 * lx) * 4;
    const uint32_t db = sd0 + (uint32_t)((ly * TX + 4 * lx) * 4);
    cp_async_wait<LA - 1>();
    __syncthreads();
    const int zlo = inj_lo, zhi = inj_hi;
#pragma unroll
    for (int k = 0; k < RAD; k++) win[RAD + k] = (z0 + k < G.NZ) ? step::lds(ub + (uint32_t)k * USZ) : step::zero();

    const int zs0 = G.nbl, zs1 = G.nbl + G.nz;   // planes outside the z absorbing layers
    const int warp = tid >> 5, lane = tid & 31;
    for (int zb = z0; zb < z1; zb += U) {
#pragma unroll
        for (int ph = 0; ph < U; ph++) {
            const int z = zb + ph;
            if (z >= z1) break;
            const int rel = z - z0;
            cp_async_wait<LA - 1>();
            __syncthreads();
            issue_u(z + RAD + LA);
            issue_db(z + LA);
            cp_async_commit();

            win[2 * RAD + ph] = (z + RAD < G.NZ) ? step::lds(ub + (uint32_t)((rel + RAD) & (NU - 1)) * USZ)
                                                 : step::zero();   // plane z+4
            const uint32_t az = ub + (uint32_t)(rel & (NU - 1)) * USZ;
            const P4 wl = step::lds(az - 16);
            const P4 wr = step::lds(az + 16);
            P4 yp[RAD], ym[RAD];
            if (TY > 1) {
#pragma unroll
                for (int k = 1; k <= RAD; k++) {
                    yp[k - 1] = step::lds(az + (uint32_t)(k * W * 4));
                    ym[k - 1] = step::lds(az - (uint32_t)(k * W * 4));
                }
            }
            const uint32_t adb = db + (uint32_t)(rel & (NDB - 1)) * DSZ;
            const P4 din = step::lds(adb);
            const P4 bb = step::lds(adb + TY * TX * 4);

            int e0 = 0, e1 = 0;
            if (rel >= zlo && rel <= zhi) {
                e0 = off[key0 + rel];
                e1 = off[key0 + rel + 1];
            }
            const bool inj = e1 > e0;
            if (inj) {
                // each warp sums the entries of its own columns: entry column a belongs to
                // thread (a / TX) * TXT + (a % TX) / 4, so no block barrier is needed
                *(float4 *)&sq[ly][4 * lx] = make_float4(0.f, 0.f, 0.f, 0.f);
                __syncwarp();
                for (int e = e0 + lane; e < e1; e += 32) {
                    const InjEntry E = A.inj[e];
                    if ((((E.a / TX) * TXT + (E.a % TX) / 4) >> 5) == warp)
                        atomicAdd(&(&sq[0][0])[E.a], E.w * A.tr_sign * tr[(long long)E.trace * A.tr_rs]);
                }
                __syncwarp();
            }
            if (!row_ok) continue;
            P4 dn, un;
            float sdv[4];
            step::step4<(TY > 1), WD>(&win[ph], yp, ym, wl, wr, din, bb, &sq[ly][4 * lx], inj,
                                  col_int && z >= zs0 && z < zs1, sdx, z, G, dn, un, sdv);
            if (has_pad) step::zero_pad(xc, G.NX, dn, un);   // padding columns stay zero
            const long long oz = (long long)z * PS;
            *(P4 *)(uo + oz) = un;
            *(P4 *)(dout + oz) = dn;
            if (IMG) {
                float u4[4];
                step::upk(un.a, u4[0], u4[1]);
                step::upk(un.b, u4[2], u4[3]);
                const long long p = oz + own;
                float4 h1, h0, gv;
                float4 *gi = (float4 *)(A.img + sh * A.img_ss + p);
                if (S::DBSLOT == 5 * TY * TX) {   // staged with the increment (2-D)
                    h1 = *(const float4 *)&dbring[(rel & (NDB - 1)) * S::DBSLOT + 2 * TY * TX + ly * TX + 4 * lx];
                    h0 = *(const float4 *)&dbring[(rel & (NDB - 1)) * S::DBSLOT + 3 * TY * TX + ly * TX + 4 * lx];
                    gv = *(const float4 *)&dbring[(rel & (NDB - 1)) * S::DBSLOT + 4 * TY * TX + ly * TX + 4 * lx];
                } else {
                    h1 = *(const float4 *)(A.h1 + sh * A.h_ss + p);
                    h0 = *(const float4 *)(A.h0 + sh * A.h_ss + p);
                    gv = *gi;
                }
                gv.x += A.img_scale * ((1.f + sdv[0]) * h1.x - (1.f - sdv[0]) * h0.x) * u4[0];
                gv.y += A.img_scale * ((1.f + sdv[1]) * h1.y - (1.f - sdv[1]) * h0.y) * u4[1];
                gv.z += A.img_scale * ((1.f + sdv[2]) * h1.z - (1.f - sdv[2]) * h0.z) * u4[2];
                gv.w += A.img_scale * ((1.f + sdv[3]) * h1.w - (1.f - sdv[3]) * h0.w) * u4[3];
                *gi = gv;
            }
        }
        // slide the window by U planes
#pragma unroll
        for (int k = 0; k < 2 * RAD; k++) win[k] = win[k + U];
    }
    cp_async_wait<0>();
}

__global__ void gather_kernel(const StencilArgs A) { gather_rows(A, blockIdx.x); }

template <int TXT, int TY, bool IMG, bool WD>
static void launch_variant(const GridDev &G, const StencilArgs &A, dim3 grid, cudaStream_t s)
{
    using S = StencilShape<TXT, TY, stencil_na<TXT, TY, IMG>()>;
    cudaFuncSetAttribute(stencil_kernel<TXT, TY, IMG, WD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    stencil_kernel<TXT, TY, IMG, WD><<<grid, S::NT, S::SMEM, s>>>(G, A);
}

template <int TXT, int TY>
static void launch_tiles(const GridDev &G, const StencilArgs &A, bool imaging, cudaStream_t s)
{
    using S = StencilShape<TXT, TY>;
    dim3 grid(stencil_tiles(G) + gather_blocks(A, S::NT), A.nshots);
    if (imaging) launch_variant<TXT, TY, true, false>(G, A, grid, s);   // exact adjoint: (u, d) form
    else if (A.wd) launch_variant<TXT, TY, false, true>(G, A, grid, s);
    else launch_variant<TXT, TY, false, false>(G, A, grid, s);
}

template <int TXT, int TY>
static int blocks_per_sm()
{
    using S = StencilShape<TXT, TY>;
    static int cached = 0;
    if (!cached) {
        cudaFuncSetAttribute(stencil_kernel<TXT, TY, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stencil_kernel<TXT, TY, false, false>, S::NT, S::SMEM) != cudaSuccess || n < 1)
            n = 1;
        cached = n;
    }
    return cached;
}

int stencil_choose_tx(const GridDev &G)
{
    if (G.ndim == 3) return T3X;
    if (const char *e = getenv("WP_STENCIL_TX")) {
        const int v = atoi(e);
        if (v == 128 || v == 256) return v;
    }
    // the narrower tile only when it pads the row less (halos and blocks cost less wide)
    const int pad128 = (G.NX + 127) / 128 * 128 - G.NX, pad256 = (G.NX + 255) / 256 * 256 - G.NX;
    return pad128 < pad256 ? 128 : 256;
}

int stencil_blocks_per_sm(const GridDev &G)
{
    if (G.ndim == 3) return blocks_per_sm<T3TX, T3Y>();
    return G.tx == 128 ? blocks_per_sm<32, 1>() : blocks_per_sm<64, 1>();
}

int device_sm_count()
{
    static int sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (!sms[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 148;
        sms[dev] = n;
    }
    return sms[dev];
}

cudaError_t launch_stencil(const GridDev &G, const StencilArgs &A, bool imaging, cudaStream_t s)
{
    if (G.ndim == 2 && G.tx != 128 && G.tx != 256) return cudaErrorInvalidValue;
    if (G.ndim == 3 && G.tx != T3X) return cudaErrorInvalidValue;
    cudaEvent_t ev = prof_begin(PROF_STENCIL, s);
    if (G.ndim == 3) launch_tiles<T3TX, T3Y>(G, A, imaging, s);
    else if (G.tx == 128) launch_tiles<32, 1>(G, A, imaging, s);
    else launch_tiles<64, 1>(G, A, imaging, s);
    prof_end(PROF_STENCIL, ev, s);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_gather(const GridDev &G, const StencilArgs &A, cudaStream_t s)
{
    (void)G;
    dim3 grid(gather_blocks(A, 256), A.nshots);
    if (grid.x == 0) return cudaSuccess;
    gather_kernel<<<grid, 256, 0, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
