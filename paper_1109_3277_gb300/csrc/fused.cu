// Fused fluid step (§2 of Günther et al., arXiv:1109.3277): ψ = 1 - exp(-ρ)
// from the populations, the Shan–Chen force (Eq. 3), the shifted-velocity
// BGK collision (Eq. 2) and push streaming (Eq. 1) with halfway bounce-back,
// in one pass over the populations.
//
// A CTA owns a TX x TY column of nodes and walks a chunk of z planes.  For
// every plane it computes ρ and ψ of the tile plus a one-node halo into a
// three-plane ring in shared memory (solid nodes take the shell ψ written by
// the shell-fill kernel), together with the moments of its own nodes.  The
// own nodes' populations are read from HBM once, in that density pass, and
// staged in shared memory (two plane buffers) for the collision one plane
// later; the force at a node reads its 18 neighbours' ψ from shared memory.
// The halo densities re-read neighbouring tiles' populations, which their
// own CTAs are streaming through L2 at the same time.
//
// Links into particle nodes get the moving bounce-back term C (Eq. 4) in
// registers as they are reflected.  Their momentum exchange (Eq. 5) and
// torque are summed per particle in 64-bit fixed point (2^-40 units): each
// FP32 link term is rounded once to an integer, and integer atomics in a
// per-CTA shared-memory table, then in the per-particle totals, add them
// exactly, so the sums do not depend on the order the links are met in.
#include "lbe_internal.cuh"

namespace lbe {

namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int HX = TX + 2, HY = TY + 2, HN = HX * HY, NHALO = HN - NT;

template <class S>
__device__ __forceinline__ const typename S::T *cslot(const typename S::T *f, const Lat &L, int c, int i)
{
    return f + (size_t)(c * Q + i) * (size_t)L.S;
}
template <class S>
__device__ __forceinline__ typename S::T *wslot(typename S::T *f, const Lat &L, int c, int i)
{
    return f + (size_t)(c * Q + i) * (size_t)L.S;
}

__device__ __forceinline__ int wrapc(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

constexpr int TAB = 128;       // per-CTA particle table (power of two)

__constant__ int c_x[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__constant__ int c_y[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__constant__ int c_z[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

// Dynamic shared memory layout (bytes).
template <class S>
struct Smem {
    static constexpr size_t fbuf = 0;                                          // T [2][2Q][NT]
    static constexpr size_t sps = fbuf + 2 * 2 * Q * NT * sizeof(typename S::T);  // float [3][2][HN]
    static constexpr size_t smo = sps + 3 * 2 * HN * sizeof(float);             // float [2][5][NT]
    static constexpr size_t tacc = smo + 2 * 5 * NT * sizeof(float);           // int64 [6][TAB]
    static constexpr size_t tid_ = tacc + 6 * TAB * sizeof(long long);          // int [TAB]
    static constexpr size_t sow = tid_ + TAB * sizeof(int);                     // int [3][HN] owners
    static constexpr size_t lq = sow + 3 * HN * sizeof(int);                    // uint16 [NT] link nodes
    static constexpr size_t lpm = lq + NT * sizeof(unsigned short);             // uint32 [NT] link masks
    static constexpr size_t lqn = lpm + NT * sizeof(uint32_t);                  // int
    static constexpr size_t sty = lqn + 16;                                      // uint8 [3][HN]
    static constexpr size_t bytes = sty + 3 * HN;
};

// FP32 value to 64-bit fixed point in units of 2^-40 (two's complement in an
// unsigned word, so that wrap-around addition is exact); |v| is clamped to
// 2^22, far beyond any link term.
__device__ __forceinline__ unsigned long long to_fixed(float v)
{
    v = fminf(fmaxf(v, -4194304.f), 4194304.f);
    return (unsigned long long)__float2ll_rn(v * 1099511627776.f);
}

// Slot of particle p in the CTA's table (linear probing, at most TAB
// probes); -1 when the table is full.
__device__ __forceinline__ int tab_slot(int *ids, int p)
{
    int h = (int)(((unsigned)p * 2654435761u) >> 25) & (TAB - 1);
    for (int k = 0; k < TAB; k++) {
        int cur = *(volatile int *)&ids[h];
        if (cur == p) return h;
        if (cur == -1) {
            int old = atomicCAS(&ids[h], -1, p);
            if (old == -1 || old == p) return h;
        }
        h = (h + 1) & (TAB - 1);
    }
    return -1;
}

// Wrapped neighbour index of a node on the lattice boundary (off the hot
// path; scalar arguments only, so that nothing is copied to local memory).
__device__ __noinline__ int wrapped_nbr(int nx, int ny, int nz, int gx, int gy, int z, int i)
{
    int x = gx + c_x[i], y = gy + c_y[i], zz = z + c_z[i];
    x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
    return x + nx * (y + ny * zz);
}

// Add this lane's fixed-point sums v[6] for particle p (or nothing, p < 0)
// to the CTA table: lanes of the warp with the same particle are combined
// first (exact integer reductions over 16/16/32-bit limbs), and one lane per
// particle does the atomics.  Must be called by all 32 lanes.
__device__ __forceinline__ void warp_add(int p, const unsigned long long v[6], const Links &lk, int *tids,
                                         unsigned long long *tacc)
{
    const unsigned grp = __match_any_sync(0xffffffffu, p);
    const int lane = threadIdx.x & 31;
    const bool leader = lane == __ffs(grp) - 1;
    unsigned long long tot[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const unsigned lo = (unsigned)v[k], hi = (unsigned)(v[k] >> 32);
        const unsigned s0 = __reduce_add_sync(grp, lo & 0xffffu);
        const unsigned s1 = __reduce_add_sync(grp, lo >> 16);
        const unsigned s2 = __reduce_add_sync(grp, hi);
        tot[k] = ((unsigned long long)s2 << 32) + ((unsigned long long)s1 << 16) + (unsigned long long)s0;
    }
    if (p < 0 || !leader) return;
    const int h = tab_slot(tids, p);
#pragma unroll
    for (int k = 0; k < 6; k++) {
        if (h >= 0)
            atomicAdd(&tacc[k * TAB + h], tot[k]);
        else
            atomicAdd(&lk.fix[6 * p + k], tot[k]);
    }
}

// All particle links of node t of the CTA's tile (plane z); t < 0: no node
// (the lane still takes part in the warp reductions).  The node's moments,
// the ψ ring and the staged populations are still in shared memory, so its
// equilibrium velocity and the post-collision populations f*_i are
// recomputed here.  The population reflected along -c_i gains
// C = 6 w_i ρ^c u_surf.(-c_i) (Eq. 4), u_surf = V + ω x r_b at the link
// midpoint r_b = node + c_i/2 - X, and the particle receives (2 f*_i + C) c_i
// and r_b x that (Eq. 5), summed in 2^-40 fixed point.
template <class S>
__device__ __forceinline__ void link_node(const Lat &L, const Links &lk, int t, uint32_t pm, int z, int x0, int y0,
                                          const typename S::T *fbuf, const float *smo, const float *sps,
                                          const int *sow, typename S::T *fout, int *tids, unsigned long long *tacc)
{
    unsigned long long acc[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    int pcur = -1;
    const int tt = t < 0 ? 0 : t;
    const int ttx = tt % TX, tty = tt / TX;
    const int lx = wrapc(x0 + ttx, L.nx), ly = wrapc(y0 + tty, L.ny);
    const int nn = lx + L.nx * (ly + L.ny * z);
    const int ec = (tty + 1) * HX + (ttx + 1);
    const int sl0 = (z + 2) % 3, sl1 = z % 3, sl2 = (z + 1) % 3;
    const int par = z & 1;
    float ue[2][3], uu[2], rho[2];
    float4 X = make_float4(0.f, 0.f, 0.f, 0.f), V = X, W = X;
    if (pm) {
        // the node's equilibrium velocity, as in the collision
        const float *mo = smo + par * 5 * NT + tt;
        rho[0] = mo[0];
        rho[1] = mo[NT];
        const float up[3] = {mo[2 * NT], mo[3 * NT], mo[4 * NT]};
        float s[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int j = 1; j < Q; j++) {
            const int slj = cz(j) < 0 ? sl0 : (cz(j) == 0 ? sl1 : sl2);
            const float *pp = sps + slj * 2 * HN + ec + cy(j) * HX + cx(j);
            const float p0 = pp[0], p1 = pp[HN];
            if (cx(j)) { s[0][0] += cx(j) * p1; s[1][0] += cx(j) * p0; }
            if (cy(j)) { s[0][1] += cy(j) * p1; s[1][1] += cy(j) * p0; }
            if (cz(j)) { s[0][2] += cz(j) * p1; s[1][2] += cz(j) * p0; }
        }
        const float pc[2] = {sps[sl1 * 2 * HN + ec], sps[sl1 * 2 * HN + HN + ec]};
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const float r = rho[c];
            const float ir = r > 0.f ? L.tau[c] / r : 0.f;
#pragma unroll
            for (int k = 0; k < 3; k++) ue[c][k] = up[k] + ir * (-L.g * pc[c] * s[c][k] + r * L.body[k]);
            uu[c] = 1.f - 1.5f * (ue[c][0] * ue[c][0] + ue[c][1] * ue[c][1] + ue[c][2] * ue[c][2]);
        }
    }
    const typename S::T *fbt = fbuf + par * 2 * Q * NT + tt;
    while (pm) {
        const int i = __ffs(pm) - 1;
        pm &= pm - 1;
        const int cxi = c_x[i], cyi = c_y[i], czi = c_z[i];
        const int sli = czi < 0 ? sl0 : (czi == 0 ? sl1 : sl2);
        const int p = sow[sli * HN + ec + cyi * HX + cxi];
        if (p != pcur) {
            if (pcur >= 0) {  // a second particle at this node: add the first directly
                const int h = tab_slot(tids, pcur);
#pragma unroll
                for (int k = 0; k < 6; k++) {
                    if (h >= 0)
                        atomicAdd(&tacc[k * TAB + h], acc[k]);
                    else
                        atomicAdd(&lk.fix[6 * pcur + k], acc[k]);
                    acc[k] = 0ull;
                }
            }
            pcur = p;
            X = lk.X32[p];
            V = lk.K32[2 * p];
            W = lk.K32[2 * p + 1];
        }
        float rx = (float)lx - X.x, ry = (float)ly - X.y, rz = (float)z - X.z;
        if (rx > 0.5f * L.nx) rx -= L.nx;
        if (rx < -0.5f * L.nx) rx += L.nx;
        if (ry > 0.5f * L.ny) ry -= L.ny;
        if (ry < -0.5f * L.ny) ry += L.ny;
        if (!L.walls) {
            if (rz > 0.5f * L.nz) rz -= L.nz;
            if (rz < -0.5f * L.nz) rz += L.nz;
        }
        rx += 0.5f * cxi;
        ry += 0.5f * cyi;
        rz += 0.5f * czi;
        const float usx = V.x + W.y * rz - W.z * ry, usy = V.y + W.z * rx - W.x * rz, usz = V.z + W.x * ry - W.y * rx;
        const float uci = usx * cxi + usy * cyi + usz * czi;
        const bool axis = i < 7;
        const float w = axis ? 1.f / 18.f : 1.f / 36.f;
        const int io = (i & 1) ? i + 1 : i - 1;
        float a = 0.f;
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const float r = rho[c];
            const float cu = cxi * ue[c][0] + cyi * ue[c][1] + czi * ue[c][2];
            const float wr = w * r;
            const float feq = wr * (uu[c] + 4.5f * cu * cu) + 3.f * wr * cu;
            const float base = axis ? L.base[c][1] : L.base[c][7];
            const float fi = S::cvt(fbt[(c * Q + i) * NT], base);
            const float fs = fi - (fi - feq) * L.itau[c];
            const float C = -6.f * wr * uci;
            S::st(fout + nn + (long long)(c * Q + io) * L.S, fs + C, base);
            a += 2.f * fs + C;
        }
        const float Fx = a * cxi, Fy = a * cyi, Fz = a * czi;
        acc[0] += to_fixed(Fx);
        acc[1] += to_fixed(Fy);
        acc[2] += to_fixed(Fz);
        acc[3] += to_fixed(ry * Fz - rz * Fy);
        acc[4] += to_fixed(rz * Fx - rx * Fz);
        acc[5] += to_fixed(rx * Fy - ry * Fx);
    }
    warp_add(pcur, acc, lk, tids, tacc);
}

// Offsets of the population arrays, per lattice, passed with the launch:
// pop[c*Q+i] = (c*Q+i)*S and push[c*Q+i] = pop[c*Q+i] + (cx + cy*nx + cz*nx*ny),
// so the address of a load or of an interior push is one add.
struct FusedOfs {
    long long pop[2 * Q];
    long long push[2 * Q];
};

template <class S>
__global__ void __launch_bounds__(NT, 3) k_fused(Lat L, const typename S::T *__restrict__ fin,
                                              typename S::T *__restrict__ fout,
                                              const float *__restrict__ psi,
                                              const uint8_t *__restrict__ type, int zc, Links lk,
                                              FusedOfs ofs)
{
    using T = typename S::T;
    extern __shared__ __align__(16) unsigned char smem[];
    T *fbuf = reinterpret_cast<T *>(smem + Smem<S>::fbuf);          // [parity][c*Q+i][tid]
    float *sps = reinterpret_cast<float *>(smem + Smem<S>::sps);    // [slot][c][e]
    float *smo = reinterpret_cast<float *>(smem + Smem<S>::smo);    // [parity][k][tid]
    uint8_t *sty = smem + Smem<S>::sty;                             // [slot][e]
    unsigned long long *tacc = reinterpret_cast<unsigned long long *>(smem + Smem<S>::tacc);  // [k][TAB]
    int *tids = reinterpret_cast<int *>(smem + Smem<S>::tid_);      // [TAB]
    int *sow = reinterpret_cast<int *>(smem + Smem<S>::sow);        // [slot][e] particle owners
    unsigned short *lq = reinterpret_cast<unsigned short *>(smem + Smem<S>::lq);  // link queue
    uint32_t *lpm = reinterpret_cast<uint32_t *>(smem + Smem<S>::lpm);  // link mask per node
    int *lqn = reinterpret_cast<int *>(smem + Smem<S>::lqn);        // queue length
    if (threadIdx.x == 0) *lqn = 0;
    for (int e = threadIdx.x; e < TAB; e += NT) {
        tids[e] = -1;
#pragma unroll
        for (int k = 0; k < 6; k++) tacc[k * TAB + e] = 0ull;
    }
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * zc, ze = min(zb + zc, L.nz);
    const int gx = wrapc(x0 + tx, L.nx), gy = wrapc(y0 + ty, L.ny);
    const bool active = (x0 + tx < L.nx) && (y0 + ty < L.ny);
    const int nxy = L.nx * L.ny;
    const int ec = (ty + 1) * HX + (tx + 1);

    // halo entry of this thread (threads tid < NHALO): top row, bottom row,
    // left column, right column of the (TX+2) x (TY+2) tile
    int he = 0, hn2 = 0;
    if (tid < NHALO) {
        int hx, hy;
        if (tid < HX) {
            hx = tid;
            hy = 0;
        } else if (tid < 2 * HX) {
            hx = tid - HX;
            hy = HY - 1;
        } else if (tid < 2 * HX + TY) {
            hx = 0;
            hy = tid - 2 * HX + 1;
        } else {
            hx = HX - 1;
            hy = tid - 2 * HX - TY + 1;
        }
        he = hy * HX + hx;
        hn2 = wrapc(x0 + hx - 1, L.nx) + L.nx * wrapc(y0 + hy - 1, L.ny);
    }
    const int own2 = gx + L.nx * gy;

    // ρ and ψ of plane zz (tile + halo) into the ring; for own nodes also
    // the moments and, when own_pops, the raw populations (plane parity).
    auto load_plane = [&](int zz, bool own_pops) {
        const int slot = (zz + 3) % 3;
        bool zin = true;
        int gz = zz;
        if (L.walls) {
            zin = zz >= 0 && zz < L.nz;
        } else {
            gz = zz < 0 ? zz + L.nz : (zz >= L.nz ? zz - L.nz : zz);
        }
        float *ps = sps + slot * 2 * HN;
        uint8_t *ts = sty + slot * HN;
        int *os = sow + slot * HN;
        {
            float p0 = 0.f, p1 = 0.f;
            uint8_t t = WALL;
            if (zin) {
                const int n = own2 + nxy * gz;
                t = type[n];
                if (t == FLUID) {
                    const int par = zz & 1;
                    T *fb = fbuf + par * 2 * Q * NT + tid;
                    const T *src = fin + n;
                    float r[2], j[2][3];
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        float v[Q];
#pragma unroll
                        for (int i = 0; i < Q; i++) {
                            const T raw = __ldg(src + ofs.pop[c * Q + i]);
                            if (own_pops) fb[(c * Q + i) * NT] = raw;
                            v[i] = S::cvt(raw, L.base[c][i]);
                        }
                        float a = v[0];
#pragma unroll
                        for (int i = 1; i < Q; i++) a += v[i];
                        r[c] = a;
                        // opposite pairs (i, i+1): c_{i+1} = -c_i
                        float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
                        for (int i = 1; i < Q; i += 2) {
                            const float d = v[i] - v[i + 1];
                            if (cx(i)) jx += cx(i) * d;
                            if (cy(i)) jy += cy(i) * d;
                            if (cz(i)) jz += cz(i) * d;
                        }
                        j[c][0] = jx;
                        j[c][1] = jy;
                        j[c][2] = jz;
                    }
                    p0 = 1.f - expf(-r[0]);
                    p1 = 1.f - expf(-r[1]);
                    if (own_pops) {
                        float *mo = smo + par * 5 * NT + tid;
                        const float den = r[0] * L.itau[0] + r[1] * L.itau[1];
                        const float iden = den > 0.f ? 1.f / den : 0.f;
                        mo[0] = r[0];
                        mo[NT] = r[1];
#pragma unroll
                        for (int k = 0; k < 3; k++) mo[(2 + k) * NT] = (j[0][k] * L.itau[0] + j[1][k] * L.itau[1]) * iden;
                    }
                } else {
                    p0 = psi[n];
                    p1 = psi[(size_t)L.N + n];
                    if (t == PART) os[ec] = (int)lk.owner[n];
                }
            }
            ps[ec] = p0;
            ps[HN + ec] = p1;
            ts[ec] = t;
        }
        if (tid < NHALO) {
            float p0 = 0.f, p1 = 0.f;
            uint8_t t = WALL;
            if (zin) {
                const int n = hn2 + nxy * gz;
                t = type[n];
                if (t == FLUID) {
                    const T *src = fin + n;
                    float r0 = 0.f, r1 = 0.f;
#pragma unroll
                    for (int i = 0; i < Q; i++) {
                        r0 += S::cvt(__ldg(src + ofs.pop[i]), L.base[0][i]);
                        r1 += S::cvt(__ldg(src + ofs.pop[Q + i]), L.base[1][i]);
                    }
                    p0 = 1.f - expf(-r0);
                    p1 = 1.f - expf(-r1);
                } else {
                    p0 = psi[n];
                    p1 = psi[(size_t)L.N + n];
                    if (t == PART) os[he] = (int)lk.owner[n];
                }
            }
            ps[he] = p0;
            ps[HN + he] = p1;
            ts[he] = t;
        }
    };

    load_plane(zb - 1, false);
    load_plane(zb, true);
    const bool xy_inner = gx >= 1 && gx <= L.nx - 2 && gy >= 1 && gy <= L.ny - 2;
    for (int z = zb; z < ze; z++) {
        load_plane(z + 1, z + 1 < ze);
        __syncthreads();
        // ring slots of planes z-1, z, z+1
        const float *pl[3] = {sps + ((z + 2) % 3) * 2 * HN, sps + (z % 3) * 2 * HN, sps + ((z + 1) % 3) * 2 * HN};
        const uint8_t *tl[3] = {sty + ((z + 2) % 3) * HN, sty + (z % 3) * HN, sty + ((z + 1) % 3) * HN};
        if (active && tl[1][ec] == FLUID) {
            const int n = own2 + nxy * z;
            const bool inner = xy_inner && z >= 1 && z <= L.nz - 2;
            const int par = z & 1;
            const float *mo = smo + par * 5 * NT + tid;
            const float rho[2] = {mo[0], mo[NT]};
            const float up[3] = {mo[2 * NT], mo[3 * NT], mo[4 * NT]};
            const T *fb = fbuf + par * 2 * Q * NT + tid;
            float s[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
            uint32_t solid = 0, part = 0;  // bit i: neighbour i is not fluid / is a particle node
#pragma unroll
            for (int i = 1; i < Q; i++) {
                const int e = ec + cy(i) * HX + cx(i);
                const float *pp = pl[cz(i) + 1];
                const float p0 = pp[e], p1 = pp[HN + e];
                const uint8_t tn = tl[cz(i) + 1][e];
                solid |= (uint32_t)(tn != FLUID) << i;
                part |= (uint32_t)(tn == PART) << i;
                if (cx(i)) { s[0][0] += cx(i) * p1; s[1][0] += cx(i) * p0; }
                if (cy(i)) { s[0][1] += cy(i) * p1; s[1][1] += cy(i) * p0; }
                if (cz(i)) { s[0][2] += cz(i) * p1; s[1][2] += cz(i) * p0; }
            }
            const float pc[2] = {pl[1][ec], pl[1][HN + ec]};
            T *dst = fout + n;
            // store of the post-collision population fs of direction i:
            // streamed to the neighbour, or reflected into slot opp(i) of
            // this node; reflections off particle nodes are left to the link
            // pass after the plane (moving bounce-back, momentum exchange)
            auto put = [&](int c, int i, float fs, float r) {
                const int ci = c * Q + i;
                if (!(solid & (1u << i))) {
                    T *q = inner ? dst + ofs.push[ci] : fout + ofs.pop[ci] + wrapped_nbr(L.nx, L.ny, L.nz, gx, gy, z, i);
                    S::st(q, fs, L.base[c][i]);
                } else if (!(part & (1u << i))) {
                    S::st(dst + ofs.pop[c * Q + opp(i)], fs, L.base[c][opp(i)]);
                }
            };
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const float r = rho[c];
                float ue[3];
                const float ir = r > 0.f ? L.tau[c] / r : 0.f;
#pragma unroll
                for (int k = 0; k < 3; k++) ue[k] = up[k] + ir * (-L.g * pc[c] * s[c][k] + r * L.body[k]);
                const float uu15 = 1.f - 1.5f * (ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2]);
                const float it = L.itau[c];

                float seq = 0.f;
                // opposite pairs share the even part of the equilibrium
#pragma unroll
                for (int i = 1; i < Q; i += 2) {
                    const float cu = cx(i) * ue[0] + cy(i) * ue[1] + cz(i) * ue[2];
                    const float wr = wgt(i) * r;
                    const float even = wr * (uu15 + 4.5f * cu * cu);
                    const float odd = 3.f * wr * cu;
                    const float fa = S::cvt(fb[(c * Q + i) * NT], L.base[c][i]);
                    const float fbv = S::cvt(fb[(c * Q + i + 1) * NT], L.base[c][i + 1]);
                    seq += 2.f * even;
                    put(c, i, fa - (fa - (even + odd)) * it, r);
                    put(c, i + 1, fbv - (fbv - (even - odd)) * it, r);
                }
                // rest population: equilibrium ρ - Σ_{i>0} f^eq_i (exact mass)
                const float f0 = S::cvt(fb[(c * Q) * NT], L.base[c][0]);
                S::st(dst + ofs.pop[c * Q], f0 - (f0 - (r - seq)) * it, L.base[c][0]);
            }
            if (part) {
                // queue this node for the link pass
                lpm[tid] = part;
                lq[atomicAdd(lqn, 1)] = (unsigned short)tid;
            }
        }
        __syncthreads();
        // Link pass: every thread takes one queued node and all its links;
        // consecutive queue entries go to different warps, so that the
        // work spreads over the whole CTA.
        const int nq = *lqn;
        if (nq > 0) {
            const int qi = (tid & 31) * (NT / 32) + (tid >> 5);
            const int t = qi < nq ? lq[qi] : -1;
            link_node<S>(L, lk, t, t >= 0 ? lpm[t] : 0u, z, x0, y0, fbuf, smo, sps, sow, fout, tids, tacc);
            __syncthreads();
        }
        if (tid == 0) *lqn = 0;
    }
    // flush the per-particle link sums of this CTA
    for (int e = threadIdx.x; e < TAB; e += NT) {
        const int p = tids[e];
        if (p < 0) continue;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            atomicAdd(&lk.fix[6 * p + k], tacc[k * TAB + e]);
            atomicAdd(&lk.fix[6 * p + 3 + k], tacc[(3 + k) * TAB + e]);
        }
    }
}

}  // namespace

#define LBE_DISPATCH(storage, CALL)                                   \
    do {                                                              \
        switch (storage) {                                            \
        case LBE_STORE_F16_OFS: { using S = StF16; CALL; } break;     \
        case LBE_STORE_BF16_OFS: { using S = StBF16; CALL; } break;   \
        default: { using S = StF32; CALL; } break;                    \
        }                                                             \
    } while (0)

int fused_zchunk(const Lat &L)
{
    // enough CTAs to fill the GPU several times over, each chunk long enough
    // that its two extra halo planes cost little
    long long cols = (long long)((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY);
    int zc = L.nz;
    while (zc > 16 && cols * ((L.nz + zc - 1) / zc) < 8 * 152) zc = (zc + 1) / 2;
    return zc;
}

template <class S>
static void launch_fused_t(const Lat &L, const void *fin, void *fout, const float *psi, const uint8_t *type,
                           const Links &lk, cudaStream_t s)
{
    static bool configured = false;  // the attribute is per function, set once per process
    if (!configured) {
        cudaFuncSetAttribute(k_fused<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Smem<S>::bytes);
        configured = true;
    }
    const int zc = fused_zchunk(L);
    dim3 grid((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY, (L.nz + zc - 1) / zc);
    FusedOfs ofs;
    for (int c = 0; c < 2; c++)
        for (int i = 0; i < Q; i++) {
            long long o = (long long)(c * Q + i) * L.S;
            ofs.pop[c * Q + i] = o;
            ofs.push[c * Q + i] = o + cx(i) + (long long)cy(i) * L.nx + (long long)cz(i) * L.nx * L.ny;
        }
    k_fused<S><<<grid, NT, Smem<S>::bytes, s>>>(L, (const typename S::T *)fin, (typename S::T *)fout, psi, type,
                                                 zc, lk, ofs);
}

void launch_fused(int storage, const Lat &L, const void *fin, void *fout, const float *psi,
                  const uint8_t *type, const Links &lk, cudaStream_t s)
{
    LBE_DISPATCH(storage, (launch_fused_t<S>(L, fin, fout, psi, type, lk, s)));
}

}  // namespace lbe
