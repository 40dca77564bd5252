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

// Dynamic shared memory layout (bytes).
template <class S>
struct Smem {
    static constexpr size_t fbuf = 0;                                          // T [2][2Q][NT]
    static constexpr size_t sps = fbuf + 2 * 2 * Q * NT * sizeof(typename S::T);  // float [3][2][HN]
    static constexpr size_t smo = sps + 3 * 2 * HN * sizeof(float);             // float [2][5][NT]
    static constexpr size_t sty = smo + 2 * 5 * NT * sizeof(float);             // uint8 [3][HN]
    static constexpr size_t bytes = sty + 3 * HN;
};

template <class S>
__global__ void __launch_bounds__(NT) k_fused(Lat L, const typename S::T *__restrict__ fin,
                                              typename S::T *__restrict__ fout,
                                              const float *__restrict__ psi,
                                              const uint8_t *__restrict__ type, int zc)
{
    using T = typename S::T;
    extern __shared__ __align__(16) unsigned char smem[];
    T *fbuf = reinterpret_cast<T *>(smem + Smem<S>::fbuf);        // [parity][c*Q+i][tid]
    float *sps = reinterpret_cast<float *>(smem + Smem<S>::sps);  // [slot][c][e]
    float *smo = reinterpret_cast<float *>(smem + Smem<S>::smo);  // [parity][k][tid]
    uint8_t *sty = smem + Smem<S>::sty;                           // [slot][e]
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * zc, ze = min(zb + zc, L.nz);
    const int gx = wrapc(x0 + tx, L.nx), gy = wrapc(y0 + ty, L.ny);
    const bool active = (x0 + tx < L.nx) && (y0 + ty < L.ny);

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
        {
            const int e = (ty + 1) * HX + (tx + 1);
            float p0 = 0.f, p1 = 0.f;
            uint8_t t = WALL;
            if (zin) {
                const int n = gx + L.nx * (gy + L.ny * gz);
                t = type[n];
                if (t == FLUID) {
                    const int par = zz & 1;
                    T *fb = fbuf + (size_t)par * 2 * Q * NT + tid;
                    float r[2], j[2][3];
#pragma unroll
                    for (int c = 0; c < 2; c++) {
                        float a = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
                        for (int i = 0; i < Q; i++) {
                            const T raw = __ldg(cslot<S>(fin, L, c, i) + n);
                            if (own_pops) fb[(c * Q + i) * NT] = raw;
                            const float v = S::cvt(raw, L.base[c][i]);
                            a += v;
                            if (cx(i)) jx += cx(i) * v;
                            if (cy(i)) jy += cy(i) * v;
                            if (cz(i)) jz += cz(i) * v;
                        }
                        r[c] = a;
                        j[c][0] = jx;
                        j[c][1] = jy;
                        j[c][2] = jz;
                    }
                    p0 = 1.f - expf(-r[0]);
                    p1 = 1.f - expf(-r[1]);
                    if (own_pops) {
                        float *mo = smo + (size_t)par * 5 * NT + tid;
                        const float den = r[0] * L.itau[0] + r[1] * L.itau[1];
                        mo[0] = r[0];
                        mo[NT] = r[1];
#pragma unroll
                        for (int k = 0; k < 3; k++)
                            mo[(2 + k) * NT] = den > 0.f ? (j[0][k] * L.itau[0] + j[1][k] * L.itau[1]) / den : 0.f;
                    }
                } else {
                    p0 = psi[n];
                    p1 = psi[(size_t)L.N + n];
                }
            }
            sps[(slot * 2 + 0) * HN + e] = p0;
            sps[(slot * 2 + 1) * HN + e] = p1;
            sty[slot * HN + e] = t;
        }
        // halo ring: top row, bottom row, left column, right column
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
            const int e = hy * HX + hx;
            float p0 = 0.f, p1 = 0.f;
            uint8_t t = WALL;
            if (zin) {
                const int hxg = wrapc(x0 + hx - 1, L.nx), hyg = wrapc(y0 + hy - 1, L.ny);
                const int n = hxg + L.nx * (hyg + L.ny * gz);
                t = type[n];
                if (t == FLUID) {
                    float r0 = 0.f, r1 = 0.f;
#pragma unroll
                    for (int i = 0; i < Q; i++) {
                        r0 += S::ld(cslot<S>(fin, L, 0, i) + n, L.base[0][i]);
                        r1 += S::ld(cslot<S>(fin, L, 1, i) + n, L.base[1][i]);
                    }
                    p0 = 1.f - expf(-r0);
                    p1 = 1.f - expf(-r1);
                } else {
                    p0 = psi[n];
                    p1 = psi[(size_t)L.N + n];
                }
            }
            sps[(slot * 2 + 0) * HN + e] = p0;
            sps[(slot * 2 + 1) * HN + e] = p1;
            sty[slot * HN + e] = t;
        }
    };

    load_plane(zb - 1, false);
    load_plane(zb, true);
    const int xs[3] = {gx == 0 ? L.nx - 1 : gx - 1, gx, gx == L.nx - 1 ? 0 : gx + 1};
    const int ys[3] = {gy == 0 ? L.ny - 1 : gy - 1, gy, gy == L.ny - 1 ? 0 : gy + 1};
    const int ec = (ty + 1) * HX + (tx + 1);
    for (int z = zb; z < ze; z++) {
        load_plane(z + 1, z + 1 < ze);
        __syncthreads();
        const int sc = z % 3;
        if (active && sty[sc * HN + ec] == FLUID) {
            const int n = gx + L.nx * (gy + L.ny * z);
            int zs[3];
            if (L.walls) {
                zs[0] = z - 1;
                zs[2] = z + 1;
            } else {
                zs[0] = z == 0 ? L.nz - 1 : z - 1;
                zs[2] = z == L.nz - 1 ? 0 : z + 1;
            }
            zs[1] = z;
            const int par = z & 1;
            const float *mo = smo + (size_t)par * 5 * NT + tid;
            const float rho[2] = {mo[0], mo[NT]};
            const float up[3] = {mo[2 * NT], mo[3 * NT], mo[4 * NT]};
            const T *fb = fbuf + (size_t)par * 2 * Q * NT + tid;
            float s[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
            uint32_t solid = 0;  // bit i: neighbour i is not fluid
#pragma unroll
            for (int i = 1; i < Q; i++) {
                const int sl = (z + cz(i) + 3) % 3;
                const int e = (ty + 1 + cy(i)) * HX + (tx + 1 + cx(i));
                const float p0 = sps[(sl * 2 + 0) * HN + e], p1 = sps[(sl * 2 + 1) * HN + e];
                if (sty[sl * HN + e] != FLUID) solid |= 1u << i;
                if (cx(i)) { s[0][0] += cx(i) * p1; s[1][0] += cx(i) * p0; }
                if (cy(i)) { s[0][1] += cy(i) * p1; s[1][1] += cy(i) * p0; }
                if (cz(i)) { s[0][2] += cz(i) * p1; s[1][2] += cz(i) * p0; }
            }
            const float pc[2] = {sps[(sc * 2 + 0) * HN + ec], sps[(sc * 2 + 1) * HN + ec]};
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const float r = rho[c];
                float ue[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const float F = -L.g * pc[c] * s[c][k] + r * L.body[k];
                    ue[k] = r > 0.f ? up[k] + L.tau[c] * F / r : up[k];
                }
                const float uu = ue[0] * ue[0] + ue[1] * ue[1] + ue[2] * ue[2];
                const float it = L.itau[c];
                float seq = 0.f;
#pragma unroll
                for (int i = 1; i < Q; i++) {
                    const float fi = S::cvt(fb[(c * Q + i) * NT], L.base[c][i]);
                    const float cu = cx(i) * ue[0] + cy(i) * ue[1] + cz(i) * ue[2];
                    const float feq = wgt(i) * r * (1.f + 3.f * cu + 4.5f * cu * cu - 1.5f * uu);
                    seq += feq;
                    const float fs = fi - (fi - feq) * it;
                    if (!(solid & (1u << i))) {
                        const int m = xs[cx(i) + 1] + L.nx * (ys[cy(i) + 1] + L.ny * zs[cz(i) + 1]);
                        S::st(wslot<S>(fout, L, c, i) + m, fs, L.base[c][i]);
                    } else {
                        S::st(wslot<S>(fout, L, c, opp(i)) + n, fs, L.base[c][opp(i)]);
                    }
                }
                // rest population: equilibrium ρ - Σ_{i>0} f^eq_i (exact mass)
                const float f0 = S::cvt(fb[(c * Q) * NT], L.base[c][0]);
                const float fs0 = f0 - (f0 - (r - seq)) * it;
                S::st(wslot<S>(fout, L, c, 0) + n, fs0, L.base[c][0]);
            }
        }
        __syncthreads();
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
                           cudaStream_t s)
{
    static bool configured = false;  // the attribute is per function, set once per process
    if (!configured) {
        cudaFuncSetAttribute(k_fused<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Smem<S>::bytes);
        configured = true;
    }
    const int zc = fused_zchunk(L);
    dim3 grid((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY, (L.nz + zc - 1) / zc);
    k_fused<S><<<grid, NT, Smem<S>::bytes, s>>>(L, (const typename S::T *)fin, (typename S::T *)fout, psi, type, zc);
}

void launch_fused(int storage, const Lat &L, const void *fin, void *fout, const float *psi,
                  const uint8_t *type, cudaStream_t s)
{
    LBE_DISPATCH(storage, (launch_fused_t<S>(L, fin, fout, psi, type, s)));
}

}  // namespace lbe
