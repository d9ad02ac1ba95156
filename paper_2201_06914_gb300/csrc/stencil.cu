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
//     block adds the entries of its (tile, plane) keys from a CSR table in shared memory,
//     so no atomics reach global memory;
//   - recording d = R u^n of the input wavefield (extra blocks after the stencil tiles);
//   - the exact imaging condition of Eq. 2 (template flag IMG): g += u_tt^j * v^j with
//     u_tt^j rebuilt from two stored forward increments.
#include "wp_internal.cuh"

namespace wp {

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

__device__ __forceinline__ void cp_async16(uint32_t dst, const float *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 8th-order second difference in pairwise form sum_k c_k ((u[+k] + u[-k]) - 2 u[0]):
// the neighbour pair is summed first and the centre removed per pair, which keeps the FP32
// rounding of L u close to the fully differenced form at 12 instead of 16 operations.
__device__ __forceinline__ float d2(float c, float p1, float m1, float p2, float m2, float p3,
                                    float m3, float p4, float m4)
{
    const float c2 = -2.f * c;
    float acc = WP_C1 * ((p1 + m1) + c2);
    acc = fmaf(WP_C2, (p2 + m2) + c2, acc);
    acc = fmaf(WP_C3, (p3 + m3) + c2, acc);
    acc = fmaf(WP_C4, (p4 + m4) + c2, acc);
    return acc;
}

__device__ __forceinline__ float4 lds4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

__device__ __forceinline__ float f4get(const float4 &v, int j)
{
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// Block = TXT x TY threads; thread (lx, ly) owns the 4 adjacent columns
// x = x0 + 4*lx + j (j < 4) of row y = y0 + ly, so a tile is TX = 4*TXT columns wide.  The
// block marches planes z0 .. z1-1.  Planes are staged through shared memory with 16-byte
// cp.async copies (zero-filled outside the grid): a ring of NU = LA + 9 u tiles (with x/y
// halos; the nine planes z-4 .. z+4 of the stencil plus LA planes in flight) and a ring of
// NDB = LA + 1 tiles holding the increment and dt^2/m.  One barrier per plane.
template <int TXT, int TY>
struct StencilShape {
    static constexpr int TX = 4 * TXT;
    static constexpr int HY = TY > 1 ? RAD : 0;
    static constexpr int NT = TXT * TY;
    static constexpr int W = TX + 2 * RAD;
    static constexpr int H = TY + 2 * HY;
    static constexpr int LA = TY > 1 ? 3 : 4;
    static constexpr int NU = 16;   // >= LA + 9; a power of two so slots are masks
    static constexpr int NDB = 8;   // >= LA + 1
    static constexpr int USLOT = H * W;           // floats
    static constexpr int DBSLOT = 2 * TY * TX;    // floats
    static constexpr int UCH = USLOT / 4;         // 16-byte chunks per u tile
    static constexpr int DBCH = DBSLOT / 4;
    static constexpr int UK = (UCH + NT - 1) / NT;    // u chunks per thread
    static constexpr int DK = (DBCH + NT - 1) / NT;   // increment/model chunks per thread
    static constexpr size_t SMEM = (size_t)(NU * USLOT + NDB * DBSLOT) * sizeof(float);
};

template <int TXT, int TY, bool IMG>
__global__ void __launch_bounds__(TXT *TY, (TY > 1 ? 2 : 3)) stencil_kernel(const GridDev G, const StencilArgs A)
{
    using S = StencilShape<TXT, TY>;
    constexpr int TX = S::TX, HY = S::HY, W = S::W, NT = S::NT, LA = S::LA;
    extern __shared__ float4 smem4[];
    float *uring = (float *)smem4;
    float *dbring = uring + S::NU * S::USLOT;
    __shared__ float sq[2][TY][TX];

    const int ntx = (G.NX + TX - 1) / TX, nty = (G.NY + TY - 1) / TY;
    const int ntiles = ntx * nty * ((G.NZ + G.tz - 1) / G.tz);
    if ((int)blockIdx.x >= ntiles) {
        gather_block(A, blockIdx.x - ntiles);
        return;
    }
    const int tid = threadIdx.x, tile = blockIdx.x;
    const long long sh = blockIdx.y;
    const int lx = tid % TXT, ly = tid / TXT;
    const int x0 = (tile % ntx) * TX, y0 = ((tile / ntx) % nty) * TY;
    const int z0 = (tile / (ntx * nty)) * G.tz, z1 = min(z0 + G.tz, G.NZ);
    const int NXp = G.NXp, PS = G.NXp * G.NY;
    const float *__restrict__ u = A.u_in + sh * A.u_in_ss;
    const float *__restrict__ dinp = A.d_in + sh * A.d_in_ss;
    const float *__restrict__ bp = A.b;
    float *__restrict__ uo = A.u_out + sh * A.u_out_ss;
    float *__restrict__ dout = A.d_out + sh * A.d_out_ss;

    // Copy descriptors of this thread (fixed across planes): shared-memory byte offset,
    // in-plane global offset, and whether the chunk lies inside the grid in x/y.
    int us[S::UK], ug[S::UK];
    bool uv[S::UK];
#pragma unroll
    for (int k = 0; k < S::UK; k++) {
        const int c = tid + k * NT;
        const int r = c / (W / 4), k4 = c % (W / 4);
        const int x = x0 - RAD + 4 * k4, y = y0 - HY + r;
        uv[k] = c < S::UCH && x >= 0 && x < NXp && y >= 0 && y < G.NY;
        us[k] = (r * W + 4 * k4) * 4;
        ug[k] = uv[k] ? y * NXp + x : 0;
    }
    int ds[S::DK], dg[S::DK];
    bool dv[S::DK], dis_b[S::DK];
#pragma unroll
    for (int k = 0; k < S::DK; k++) {
        const int c = tid + k * NT;
        const int a = c / (TY * TX / 4), rem = c % (TY * TX / 4);
        const int r = rem / (TX / 4), k4 = rem % (TX / 4);
        const int x = x0 + 4 * k4, y = y0 + r;
        dv[k] = c < S::DBCH && x < NXp && y < G.NY;
        dis_b[k] = a == 1;
        ds[k] = (a * TY * TX + r * TX + 4 * k4) * 4;
        dg[k] = dv[k] ? y * NXp + x : 0;
    }
    const uint32_t su0 = (uint32_t)__cvta_generic_to_shared(uring);
    const uint32_t sd0 = (uint32_t)__cvta_generic_to_shared(dbring);
    static_assert((S::NU & (S::NU - 1)) == 0 && S::NU >= LA + 9, "u ring");
    static_assert((S::NDB & (S::NDB - 1)) == 0 && S::NDB >= LA + 1, "db ring");
    auto issue_u = [&](int k) {
        const uint32_t base = su0 + (uint32_t)((k & (S::NU - 1)) * S::USLOT * 4);
        const bool kin = k >= 0 && k < G.NZ;
#pragma unroll
        for (int q = 0; q < S::UK; q++)
            if (tid + q * NT < S::UCH)
                cp_async16(base + us[q], u + (kin && uv[q] ? k * PS + ug[q] : 0), kin && uv[q]);
    };
    auto issue_db = [&](int k) {
        const uint32_t base = sd0 + (uint32_t)((k & (S::NDB - 1)) * S::DBSLOT * 4);
        const bool kin = k < z1;
#pragma unroll
        for (int q = 0; q < S::DK; q++)
            if (tid + q * NT < S::DBCH) {
                const bool ok = kin && dv[q];
                const float *src = dis_b[q] ? bp : dinp;
                cp_async16(base + ds[q], src + (ok ? k * PS + dg[q] : 0), ok);
            }
    };

    const int *off = A.inj ? A.inj_off + sh * ((long long)ntiles * G.tz + 1) : nullptr;
    const bool tile_inj = off && off[(long long)tile * G.tz] < off[(long long)tile * G.tz + (z1 - z0)];
    const float *tr = tile_inj ? A.traces + sh * A.tr_ss + (long long)A.step * A.tr_ts : nullptr;
    const bool interior_xy = x0 >= G.nbl && x0 + TX <= G.nbl + G.nx &&
                             (TY == 1 || (y0 >= G.nbl && y0 + TY <= G.nbl + G.ny));
    const int gy = y0 + ly, xc = x0 + 4 * lx;
    const bool row_ok = gy < G.NY && xc < NXp;   // this thread's float4 lies in the field
    float sdx[4];
#pragma unroll
    for (int j = 0; j < 4; j++)
        sdx[j] = damp_term(xc + j, G.nx, G.nbl, G.hs0x, G.inv_nbl) +
                 (TY > 1 ? damp_term(gy, G.ny, G.nbl, G.hs0y, G.inv_nbl) : 0.f);

    // Prologue: group g (g < LA) holds u plane z0+4+g and increment/model plane z0+g;
    // group 0 also holds the u planes z0-4 .. z0+3.
    for (int k = z0 - RAD; k < z0 + RAD; k++) issue_u(k);
#pragma unroll
    for (int g = 0; g < LA; g++) {
        issue_u(z0 + RAD + g);
        issue_db(z0 + g);
        cp_async_commit();
    }

    const uint32_t ucol = (uint32_t)(RAD + 4 * lx) * 4;   // byte offset of the own float4 in a u row
    const bool has_pad = x0 + TX > G.NX;                   // tile reaches the padding columns
    for (int z = z0; z < z1; z++) {
        const int buf = (z - z0) & 1;
        cp_async_wait<LA - 1>();
        __syncthreads();
        issue_u(z + LA + RAD);
        issue_db(z + LA);
        cp_async_commit();

        // 32-bit shared addresses of the own float4 in the u tiles of planes z-4 .. z+4
        const uint32_t rowb = (uint32_t)((ly + HY) * W * 4) + ucol;
        auto ua = [&](int k) { return su0 + (uint32_t)((k & (S::NU - 1)) * (S::USLOT * 4)) + rowb; };
        const uint32_t az = ua(z);
        const float4 cc = lds4(az);
        const float4 wl = lds4(az - 16);
        const float4 wr = lds4(az + 16);
        float4 zp[RAD], zm[RAD], yp[RAD], ym[RAD];
#pragma unroll
        for (int k = 1; k <= RAD; k++) {
            zp[k - 1] = lds4(ua(z + k));
            zm[k - 1] = lds4(ua(z - k));
            if (TY > 1) {
                yp[k - 1] = lds4(az + (uint32_t)(k * W * 4));
                ym[k - 1] = lds4(az - (uint32_t)(k * W * 4));
            }
        }
        const uint32_t adb = sd0 + (uint32_t)((z & (S::NDB - 1)) * (S::DBSLOT * 4) + (ly * TX + 4 * lx) * 4);
        const float4 din = lds4(adb);
        const float4 bb = lds4(adb + TY * TX * 4);

        int e0 = 0, e1 = 0;
        if (tile_inj) {
            const long long key = (long long)tile * G.tz + (z - z0);
            e0 = off[key];
            e1 = off[key + 1];
        }
        if (e1 > e0) {
            *(float4 *)&sq[buf][ly][4 * lx] = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
            for (int e = e0 + tid; e < e1; e += NT) {
                const InjEntry E = A.inj[e];
                atomicAdd(&(&sq[buf][0][0])[E.a], E.w * A.tr_sign * tr[(long long)E.trace * A.tr_rs]);
            }
            __syncthreads();
        }
        if (!row_ok) continue;
        const float w[12] = {wl.x, wl.y, wl.z, wl.w, cc.x, cc.y, cc.z, cc.w, wr.x, wr.y, wr.z, wr.w};
        const float sdz = damp_term(z, G.nz, G.nbl, G.hs0z, G.inv_nbl);
        const bool fast = interior_xy && sdz == 0.f;
        float un[4], dn[4], sdv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const float c = w[4 + j];
            float lap = G.ihx2 * d2(c, w[5 + j], w[3 + j], w[6 + j], w[2 + j], w[7 + j], w[1 + j],
                                    w[8 + j], w[0 + j]);
            lap += G.ihz2 * d2(c, f4get(zp[0], j), f4get(zm[0], j), f4get(zp[1], j), f4get(zm[1], j),
                               f4get(zp[2], j), f4get(zm[2], j), f4get(zp[3], j), f4get(zm[3], j));
            if (TY > 1)
                lap += G.ihy2 * d2(c, f4get(yp[0], j), f4get(ym[0], j), f4get(yp[1], j),
                                   f4get(ym[1], j), f4get(yp[2], j), f4get(ym[2], j),
                                   f4get(yp[3], j), f4get(ym[3], j));
            if (e1 > e0) lap += sq[buf][ly][4 * lx + j];
            const float a = f4get(bb, j) * lap;
            const float di = f4get(din, j);
            float sd = 0.f, d;
            if (fast) {
                d = di + a;
            } else {
                sd = sdx[j] + sdz;
                d = (sd == 0.f) ? di + a : ((1.f - sd) * di + a) * __frcp_rn(1.f + sd);
            }
            const bool col = !has_pad || xc + j < G.NX;   // padding columns stay zero
            dn[j] = col ? d : 0.f;
            un[j] = col ? c + d : 0.f;
            sdv[j] = sd;
        }
        const int p = z * PS + gy * NXp + xc;
        *(float4 *)(uo + p) = make_float4(un[0], un[1], un[2], un[3]);
        *(float4 *)(dout + p) = make_float4(dn[0], dn[1], dn[2], dn[3]);
        if (IMG) {
            const float4 h1 = *(const float4 *)(A.h1 + sh * A.h_ss + p);
            const float4 h0 = *(const float4 *)(A.h0 + sh * A.h_ss + p);
            float4 *gi = (float4 *)(A.img + sh * A.img_ss + p);
            float4 gv = *gi;
            gv.x += A.img_scale * ((1.f + sdv[0]) * h1.x - (1.f - sdv[0]) * h0.x) * un[0];
            gv.y += A.img_scale * ((1.f + sdv[1]) * h1.y - (1.f - sdv[1]) * h0.y) * un[1];
            gv.z += A.img_scale * ((1.f + sdv[2]) * h1.z - (1.f - sdv[2]) * h0.z) * un[2];
            gv.w += A.img_scale * ((1.f + sdv[3]) * h1.w - (1.f - sdv[3]) * h0.w) * un[3];
            *gi = gv;
        }
    }
    cp_async_wait<0>();
}

__global__ void gather_kernel(const StencilArgs A) { gather_block(A, blockIdx.x); }

template <int TXT, int TY>
static void launch_tiles(const GridDev &G, const StencilArgs &A, bool imaging, cudaStream_t s)
{
    using S = StencilShape<TXT, TY>;
    const int ng = A.do_gather ? (A.nrec + S::NT - 1) / S::NT : 0;
    dim3 grid(stencil_tiles(G) + ng, A.nshots);
    if (imaging) {
        cudaFuncSetAttribute(stencil_kernel<TXT, TY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        stencil_kernel<TXT, TY, true><<<grid, S::NT, S::SMEM, s>>>(G, A);
    } else {
        cudaFuncSetAttribute(stencil_kernel<TXT, TY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        stencil_kernel<TXT, TY, false><<<grid, S::NT, S::SMEM, s>>>(G, A);
    }
}

cudaError_t launch_stencil(const GridDev &G, const StencilArgs &A, bool imaging, cudaStream_t s)
{
    cudaEvent_t ev = prof_begin(PROF_STENCIL, s);
    if (G.ndim == 2) launch_tiles<T2TX, T2Y>(G, A, imaging, s);
    else launch_tiles<T3TX, T3Y>(G, A, imaging, s);
    prof_end(PROF_STENCIL, ev, s);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_gather(const GridDev &G, const StencilArgs &A, cudaStream_t s)
{
    (void)G;
    dim3 grid((A.nrec + 255) / 256, A.nshots);
    gather_kernel<<<grid, 256, 0, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
