// Fused fluid step (§2 of Günther et al., arXiv:1109.3277): the Shan–Chen
// force (Eq. 3), the shifted-velocity BGK collision (Eq. 2) and push
// streaming (Eq. 1) with halfway bounce-back, in one pass over the
// populations.
//
// A CTA owns a TX x TY column of nodes and walks a chunk of z planes.  The
// populations of its nodes in a plane are staged in shared memory, two
// planes deep: while the warps collide plane z, the next plane is on its way
// into the other stage, as one TMA tensor copy (a 32 x 8 x 38-slot box of
// the population array, completion on an mbarrier) where the lattice's row
// pitch allows it, else by per-thread loads.  ψ of the tile and a one-node
// halo (written by the density kernel on fluid nodes, by the shell fill on
// solid nodes) goes into a four-slot ring of planes; the force at a node
// reads its 18 neighbours' ψ from the ring.  Moments, force, collision and
// the stores of one node run in one thread, on (red, blue) pairs.
//
// Populations streaming into a wall or particle node are reflected into the
// opposite slot of their own node (halfway bounce-back).  For particle
// nodes the moving-boundary term and the momentum exchange are added
// afterwards by the link kernel.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "lbe_internal.cuh"

namespace lbe {

namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int HX = TX + 2, HY = TY + 2, HN = HX * HY, NHALO = HN - NT;

__device__ __forceinline__ int wrapc(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Dynamic shared memory layout (bytes from a 128-byte aligned base).
template <class S>
struct Smem {
    // CTAs per SM the kernels are compiled for: three at 16 bit (51 KB of
    // shared memory each, 80 registers per thread), two in FP32 (90 KB each)
    static constexpr int CTAS = sizeof(typename S::T) == 2 ? 3 : 2;
    static constexpr size_t plane = 2 * Q * NT * sizeof(typename S::T);  // one staged plane
    static constexpr size_t stage = 0;                                   // T [2][2Q][NT]
    static constexpr size_t sps = stage + 2 * plane;                     // float2 [4][HN] (ψ_b, ψ_r)
    static constexpr size_t sty = sps + 4 * HN * sizeof(float2);         // uint8 [4][HN]
    static constexpr size_t bar = (sty + 4 * HN + 15) / 16 * 16;          // uint64 [2] mbarriers
    static constexpr size_t bytes = bar + 2 * sizeof(unsigned long long) + 128;  // + alignment slack
};

__device__ __forceinline__ unsigned char *align128(unsigned char *p)
{
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 127) & ~uintptr_t(127));
}

// ---- TMA and mbarrier (PTX) -------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(unsigned long long *b)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}

// make barrier initialisation visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// order this thread's earlier shared-memory accesses before later TMA writes
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with this parity; false if it has not completed
// within the iteration limit (each try may suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity)
{
    for (int k = 0; k < (1 << 22); k++)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

// One plane of the tile: the box (x0, y0, z, slot 0) of size 32 x 8 x 1 x 38
// of the 4D population tensor into shared memory, completing on b.
__device__ __forceinline__ void tma_plane(void *dst, const CUtensorMap *map, int x0, int y0, int z,
                                          unsigned long long *b)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x0), "r"(y0), "r"(z), "r"(0), "r"(smem_u32(b))
        : "memory");
}

// ---- node arithmetic ------------------------------------------------------
// Every product or sum that rounds is written with a round-to-nearest
// intrinsic (which the compiler never contracts), so that each kernel that
// inlines these computes the same bits: the single-lattice and the batched
// fused kernels agree exactly.  Products with the lattice velocities c_i
// (components 0 or ±1) are exact and stay plain.

// The two components go through the same node arithmetic, so it is done on
// (red, blue) pairs with the paired FP32 instructions (add, multiply and
// fused multiply-add on two lanes, each rounded to nearest like its scalar
// form): every component's result has the bits of the scalar sequence.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Equilibrium velocities of both components, u' + (τ_c/ρ_c) F^c with the
// Shan–Chen force F^c = -g ψ^c s^c + ρ^c g_body (Eq. 3), and -1.5 u·u.
__device__ __forceinline__ void eq_velocity(const Lat &L, float2 r, float2 pc, const float2 s[3], const float up[3],
                                            float2 ue[3], float2 &um15)
{
    const float2 ir = make_float2(r.x > 0.f ? __fdiv_rn(L.tau[0], r.x) : 0.f,
                                  r.y > 0.f ? __fdiv_rn(L.tau[1], r.y) : 0.f);
    const float2 gp = mul2(dup2(-L.g), pc);
#pragma unroll
    for (int k = 0; k < 3; k++) ue[k] = fma2(ir, fma2(gp, s[k], mul2(r, dup2(L.body[k]))), dup2(up[k]));
    const float2 uu = fma2(ue[0], ue[0], fma2(ue[1], ue[1], mul2(ue[2], ue[2])));
    um15 = mul2(dup2(-1.5f), uu);
}

// f^eq_i = w_i ρ (1 + 3 c·u + 4.5 (c·u)^2 - 1.5 u·u) relative to the stored
// quantity's base w_i ρ_ref: even part w_i (ρ (4.5 (c·u)^2 - 1.5 u·u) + Δρ)
// with Δρ = ρ - ρ_ref (for FP32 storage ρ_ref = 0, Δρ = ρ), odd part
// 3 w_i ρ c·u (w3r = 3 w_i ρ comes per weight).
__device__ __forceinline__ void feq_parts(float w, float2 r, float2 dr, float2 w3r, float2 cu, float2 um15,
                                          float2 &even, float2 &odd)
{
    even = mul2(dup2(w), fma2(r, fma2(mul2(dup2(4.5f), cu), cu, um15), dr));
    odd = mul2(w3r, cu);
}

// BGK relaxation f + (f^eq - f)/τ.
__device__ __forceinline__ float2 relax(float2 f, float2 feq, float2 it) { return fma2(sub2(feq, f), it, f); }

// One tile (column bx, by, z chunk bz) of one lattice.  TMA: the planes
// arrive as tensor copies described by *tmap; otherwise each thread loads
// its node's populations.  Returns false if a copy never completed (the
// lattice's status word records it).
template <class S, bool TMA, bool R32>
__device__ __forceinline__ bool fused_tile(const Lat &L, const typename S::T *__restrict__ fin,
                                           typename S::T *__restrict__ fout, const float *__restrict__ rho,
                                           const float *__restrict__ psi, const uint8_t *__restrict__ type, int zc,
                                           const FusedOfs &ofs, const CUtensorMap *tmap, int bx, int by, int bz,
                                           unsigned char *smem)
{
    using T = typename S::T;
    T *stage = reinterpret_cast<T *>(smem + Smem<S>::stage);        // [stage][c*Q+i][tid]
    float2 *sps = reinterpret_cast<float2 *>(smem + Smem<S>::sps);  // [slot][e]
    uint8_t *sty = smem + Smem<S>::sty;                             // [slot][e]
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem + Smem<S>::bar);
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = bx * TX, y0 = by * TY;
    const int zb = bz * zc, ze = min(zb + zc, L.nz);
    const int gx = wrapc(x0 + tx, L.nx), gy = wrapc(y0 + ty, L.ny);
    const bool active = (x0 + tx < L.nx) && (y0 + ty < L.ny);
    const int nxy = L.nx * L.ny;
    const int ec = (ty + 1) * HX + (tx + 1);

    // halo entry h of this thread: top row, bottom row, left column, right
    // column of the (TX+2) x (TY+2) tile; threads 2h and 2h+1 take the two
    // components of entry h
    const int h = tid >> 1, hc = tid & 1;
    int he = 0, hn2 = 0;
    if (h < NHALO) {
        int hx, hy;
        if (h < HX) {
            hx = h;
            hy = 0;
        } else if (h < 2 * HX) {
            hx = h - HX;
            hy = HY - 1;
        } else if (h < 2 * HX + TY) {
            hx = 0;
            hy = h - 2 * HX + 1;
        } else {
            hx = HX - 1;
            hy = h - 2 * HX - TY + 1;
        }
        he = hy * HX + hx;
        hn2 = wrapc(x0 + hx - 1, L.nx) + L.nx * wrapc(y0 + hy - 1, L.ny);
    }
    const int own2 = gx + L.nx * gy;

    // ψ and node type of plane zz (tile + halo) for the ring: the density
    // kernel's ψ on fluid nodes and the shell fill's on solid nodes share one
    // array, so the loads of an entry do not wait on its type; walls beyond
    // the lattice's z walls.  Loaded one plane ahead into registers, stored
    // into ring slot zz % 4 after the collision of plane zz - 2.
    struct RingVals {
        float p0, p1, ph;
        uint8_t t, th;
    };
    auto ring_load = [&](int zz) {
        RingVals v{0.f, 0.f, 0.f, WALL, WALL};
        bool zin = true;
        int gz = zz;
        if (L.walls) {
            zin = zz >= 0 && zz < L.nz;
        } else {
            // planes -1 .. nz+1: two wraps when nz = 1
            gz = zz < 0 ? zz + L.nz : zz;
            while (gz >= L.nz) gz -= L.nz;
        }
        if (zin) {
            const int n = own2 + nxy * gz;
            v.t = type[n];
            v.p0 = psi[n];
            v.p1 = psi[(size_t)L.N + n];
            if (h < NHALO) {
                const int nh = hn2 + nxy * gz;
                v.th = type[nh];
                v.ph = psi[(size_t)hc * L.N + nh];
            }
        }
        return v;
    };
    auto ring_store = [&](int zz, const RingVals &v) {
        const int slot = (zz + 4) & 3;
        float2 *ps = sps + slot * HN;
        uint8_t *ts = sty + slot * HN;
        ps[ec] = make_float2(v.p1, v.p0);  // (ψ_b, ψ_r): the partner component first
        ts[ec] = v.t;
        if (h < NHALO) {
            reinterpret_cast<float *>(ps + he)[1 - hc] = v.ph;
            if (hc == 0) ts[he] = v.th;
        }
    };

    // Populations of plane zz into stage zz & 1 (after the barrier that
    // ended the collision that last read that stage).
    auto fill = [&](int zz) {
        T *st = stage + (zz & 1) * 2 * Q * NT;
        if (TMA) {
            if (tid == 0) {
                fence_proxy_async();
                mbar_expect_tx(&bar[zz & 1], (unsigned)Smem<S>::plane);
                tma_plane(st, tmap, x0, y0, zz, &bar[zz & 1]);
            }
        } else if (active) {
            const int n = own2 + nxy * zz;
            if (type[n] == FLUID) {
                const T *src = fin + n;
#pragma unroll
                for (int ci = 0; ci < 2 * Q; ci++) st[ci * NT + tid] = __ldg(src + ofs.pop[ci]);
            }
        }
    };

    if (TMA) {
        if (tid == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_barrier_init();
        }
        __syncthreads();
    }
    fill(zb);
    ring_store(zb - 1, ring_load(zb - 1));
    ring_store(zb, ring_load(zb));
    ring_store(zb + 1, ring_load(zb + 1));
    const bool xy_inner = gx >= 1 && gx <= L.nx - 2 && gy >= 1 && gy <= L.ny - 2;
    bool ok = true;
    for (int z = zb; z < ze; z++) {
        if (z + 1 < ze) fill(z + 1);
        // the ring of plane z+2 is needed by the next collision: its loads
        // are in flight during this one
        const RingVals next = ring_load(z + 2);
        bool late = false;
        if (TMA) late = !mbar_wait(&bar[z & 1], ((z - zb) >> 1) & 1);
        if (__syncthreads_or(late)) {
            ok = false;
            break;
        }
        // ring slots of planes z-1, z, z+1
        const float2 *pl[3] = {sps + ((z + 3) & 3) * HN, sps + (z & 3) * HN, sps + ((z + 1) & 3) * HN};
        const uint8_t *tl[3] = {sty + ((z + 3) & 3) * HN, sty + (z & 3) * HN, sty + ((z + 1) & 3) * HN};
        if (active && tl[1][ec] == FLUID) {
            const int n = own2 + nxy * z;
            const bool inner = xy_inner && z >= 1 && z <= L.nz - 2;
            const T *fb = stage + (z & 1) * 2 * Q * NT + tid;
            // moments from the stored quantities d_i (δf_i in the 16-bit
            // modes, f_i in FP32): Δρ^c = Σ_i d_i, ρ^c = ρ_ref + Δρ^c, and
            // j^c = Σ_i c_i d_i (the bases cancel: Σ_i w_i c_i = 0); the
            // shifted velocity u' = Σ_c j^c/τ_c / Σ_c ρ^c/τ_c
            // (red, blue) pairs of the stored quantities of direction i
            auto ld2 = [&](int i) { return make_float2(S::raw(fb[i * NT]), S::raw(fb[(Q + i) * NT])); };
            float2 a = ld2(0), jj[3] = {dup2(0.f), dup2(0.f), dup2(0.f)};
#pragma unroll
            for (int i = 1; i < Q; i += 2) {
                // one pass over opposite pairs (i, i+1), c_{i+1} = -c_i; the
                // sum accumulates in index order
                const float2 va = ld2(i), vb = ld2(i + 1);
                a = add2(a, va);
                a = add2(a, vb);
                const float2 d = sub2(va, vb);
                if (cx(i)) jj[0] = cx(i) > 0 ? add2(jj[0], d) : sub2(jj[0], d);
                if (cy(i)) jj[1] = cy(i) > 0 ? add2(jj[1], d) : sub2(jj[1], d);
                if (cz(i)) jj[2] = cz(i) > 0 ? add2(jj[2], d) : sub2(jj[2], d);
            }
            const float2 drho = a, rho_ = add2(make_float2(L.rref[0], L.rref[1]), a);
            // 16-bit storage: the collision re-reads the stage, since keeping
            // the converted populations live in registers would spill under
            // the three-CTA register budget.  FP32 storage runs two CTAs
            // per SM (shared memory) and keeps them in registers.
            if constexpr (sizeof(T) == 2) asm volatile("" ::: "memory");
            const float den = __fmaf_rn(rho_.y, L.itau[1], __fmul_rn(rho_.x, L.itau[0]));
            const float iden = den > 0.f ? 1.f / den : 0.f;
            float up[3];
#pragma unroll
            for (int k = 0; k < 3; k++)
                up[k] = __fmul_rn(__fmaf_rn(jj[k].y, L.itau[1], __fmul_rn(jj[k].x, L.itau[0])), iden);
            // s^c = Σ_i c_i ψ^{c'}(x + c_i): the ring holds (ψ_b, ψ_r), the
            // partner of (red, blue)
            float2 s[3] = {dup2(0.f), dup2(0.f), dup2(0.f)};
            uint32_t solid = 0;  // bit i: neighbour i is not fluid
#pragma unroll
            for (int i = 1; i < Q; i++) {
                const int e = ec + cy(i) * HX + cx(i);
                const float2 pp = pl[cz(i) + 1][e];
                const uint8_t tn = tl[cz(i) + 1][e];
                solid |= (uint32_t)(tn != FLUID) << i;
                if (cx(i)) s[0] = cx(i) > 0 ? add2(s[0], pp) : sub2(s[0], pp);
                if (cy(i)) s[1] = cy(i) > 0 ? add2(s[1], pp) : sub2(s[1], pp);
                if (cz(i)) s[2] = cz(i) > 0 ? add2(s[2], pp) : sub2(s[2], pp);
            }
            const float2 pcc = pl[1][ec];
            const float2 pc = make_float2(pcc.y, pcc.x);  // own (ψ_r, ψ_b)
            T *dst = fout + n;
            // R32: stores address the node's component c from dc[c] with
            // 32-bit offsets (one wide multiply-add per address)
            T *const dc[2] = {dst, dst + (size_t)Q * (size_t)L.S};
            // A warp whose nodes are all off the lattice boundary and have
            // no solid neighbour pushes every population to its fixed
            // offset; the others select, per population, between the push
            // (with the periodic wrap of boundary nodes) and the reflection.
            const bool clean = __all_sync(__activemask(), inner && solid == 0u);
            auto collide = [&](auto clean_tag) {
                constexpr bool CLEAN = decltype(clean_tag)::value;
                // Push offsets of nodes on the lattice boundary wrap around
                // the periodic axes: corrections for c = +1 ([0]) and c = -1 ([1]).
                int wx[2] = {0, 0}, wy[2] = {0, 0}, wz[2] = {0, 0};
                if (!CLEAN && !inner) {
                    wx[0] = gx == L.nx - 1 ? -L.nx : 0;
                    wx[1] = gx == 0 ? L.nx : 0;
                    wy[0] = gy == L.ny - 1 ? -nxy : 0;
                    wy[1] = gy == 0 ? nxy : 0;
                    if (!L.walls) {  // with walls z = 0 and nz-1 are wall nodes
                        wz[0] = z == L.nz - 1 ? -L.N : 0;
                        wz[1] = z == 0 ? L.N : 0;
                    }
                }
                // store of the post-collision population fs of direction i:
                // pushed to the neighbour, or reflected into slot opp(i) of
                // this node (walls and particle nodes; the link kernel adds
                // the moving-boundary term for the latter).  Both slots have
                // the same weight, hence the same storage offset; the
                // address is a select, not a branch.
                auto put = [&](int c, int i, float fs) {
                    if (CLEAN) {
                        if constexpr (R32)
                            S::st_raw(dc[c] + ofs.push32[c * Q + i], fs);
                        else
                            S::st_raw(dst + ofs.push[c * Q + i], fs);
                    } else {
                        const int corr = (cx(i) > 0 ? wx[0] : (cx(i) < 0 ? wx[1] : 0)) +
                                         (cy(i) > 0 ? wy[0] : (cy(i) < 0 ? wy[1] : 0)) +
                                         (cz(i) > 0 ? wz[0] : (cz(i) < 0 ? wz[1] : 0));
                        if constexpr (R32) {
                            const unsigned o = ((solid >> i) & 1u) ? ofs.pop32[c * Q + opp(i)]
                                                                   : ofs.push32[c * Q + i] + (unsigned)corr;
                            S::st_raw(dc[c] + o, fs);
                        } else {
                            const long long o =
                                ((solid >> i) & 1u) ? ofs.pop[c * Q + opp(i)] : ofs.push[c * Q + i] + corr;
                            S::st_raw(dst + o, fs);
                        }
                    }
                };
                float2 ue[3], um15;
                eq_velocity(L, rho_, pc, s, up, ue, um15);
                const float2 it = make_float2(L.itau[0], L.itau[1]);
                // 3 w ρ per weight (axis 1/18, diagonal 1/36)
                const float2 w3r_a = mul2(dup2(3.f * wgt(1)), rho_), w3r_d = mul2(dup2(3.f * wgt(7)), rho_);
                float2 seq = dup2(0.f);
                // opposite pairs share the even part of the equilibrium
#pragma unroll
                for (int i = 1; i < Q; i += 2) {
                    // c·u with c components in {-1, 0, 1}: sums in x, y, z order
                    float2 cu = dup2(0.f);
                    bool first = true;
                    auto acc = [&](int ck, float2 v) {
                        if (!ck) return;
                        const float2 t = ck > 0 ? v : make_float2(-v.x, -v.y);
                        cu = first ? t : add2(cu, t);
                        first = false;
                    };
                    acc(cx(i), ue[0]);
                    acc(cy(i), ue[1]);
                    acc(cz(i), ue[2]);
                    float2 even, odd;
                    feq_parts(wgt(i), rho_, drho, i < 7 ? w3r_a : w3r_d, cu, um15, even, odd);
                    seq = add2(seq, mul2(dup2(2.f), even));
                    const float2 ra = relax(ld2(i), add2(even, odd), it);
                    const float2 rb = relax(ld2(i + 1), sub2(even, odd), it);
                    put(0, i, ra.x);
                    put(1, i, ra.y);
                    put(0, i + 1, rb.x);
                    put(1, i + 1, rb.y);
                }
                // rest population: equilibrium Δρ - Σ_{i>0} f^eq_i in the
                // stored quantity (exact mass)
                const float2 r0 = relax(ld2(0), sub2(drho, seq), it);
                S::st_raw(R32 ? dc[0] : dst + ofs.pop[0], r0.x);
                S::st_raw(R32 ? dc[1] : dst + ofs.pop[Q], r0.y);
            };
            if (clean)
                collide(std::true_type{});
            else
                collide(std::false_type{});
        } else if (active) {
            // A solid node's populations are never read (a node that a
            // particle uncovers gets f^eq in all slots), but writing them
            // keeps every sector of the output fully written: a partly
            // written sector costs a DRAM read when it leaves L2.
            T *d0 = fout + own2 + nxy * z;
#pragma unroll
            for (int ci = 0; ci < 2 * Q; ci++) d0[ofs.pop[ci]] = S::enc(0.f, 0.f);
        }
        ring_store(z + 2, next);  // slot (z+2) % 4: not one the collision read
        __syncthreads();
    }
    if (TMA) {
        if (!ok && tid == 0) {
            // let the copies in flight land (bounded) before the memory is reused
            const int n_issued = ze - zb;
            for (int st = 0; st < 2; st++) {
                const int uses = (n_issued - st + 1) / 2;  // planes zb+st, zb+st+2, ...
                if (uses > 0) mbar_wait(&bar[(zb + st) & 1], (uses - 1) & 1);
            }
            atomicOr(L.status, 1u);
        }
        __syncthreads();
        if (tid == 0) {
            mbar_inval(&bar[0]);
            mbar_inval(&bar[1]);
        }
    }
    return ok;
}

template <class S, bool TMA, bool R32>
__global__ void __launch_bounds__(NT, Smem<S>::CTAS) k_fused(Lat L, const typename S::T *__restrict__ fin,
                                              typename S::T *__restrict__ fout, const float *__restrict__ rho,
                                              const float *__restrict__ psi,
                                              const uint8_t *__restrict__ type, int zc, FusedOfs ofs,
                                              const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    fused_tile<S, TMA, R32>(L, fin, fout, rho, psi, type, zc, ofs, &tmap, blockIdx.x, blockIdx.y, blockIdx.z,
                            align128(smem_raw));
}

// Persistent multi-lattice variant: CTAs take tiles of all boxes of a batch
// from one queue (largest boxes first in the queue order set by the host).
template <class S>
__global__ void __launch_bounds__(NT, Smem<S>::CTAS) k_fused_batch(BatchIndex B, int total)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = align128(smem_raw);
    __shared__ int s_tile, s_box;
    __shared__ BoxDev sb;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_tile = atomicAdd(B.counter, 1);
            s_box = s_tile < total ? find_box(B.tile0, B.nbox, s_tile) : 0;
        }
        __syncthreads();
        const int t = s_tile;
        if (t >= total) break;
        // the box descriptor into shared memory (word copy)
        const int *src = reinterpret_cast<const int *>(B.box + s_box);
        int *dstw = reinterpret_cast<int *>(&sb);
        for (int k = threadIdx.x; k < (int)(sizeof(BoxDev) / 4); k += NT) dstw[k] = src[k];
        __syncthreads();
        const int lt = t - B.tile0[s_box];
        const int bx = lt % sb.ntx, by = (lt / sb.ntx) % sb.nty, bz = lt / (sb.ntx * sb.nty);
        const int cur = B.par[2 * s_box];
        // the tensor map stays in global memory (a TMA operand cannot be in shared memory)
        const CUtensorMap *tm = &B.box[s_box].tmap[cur];
        bool ok;
        if (sb.tma)
            ok = fused_tile<S, true, false>(sb.L, (const typename S::T *)sb.f[cur], (typename S::T *)sb.f[1 - cur], sb.rho,
                                     sb.psi, sb.type, sb.zc, sb.ofs, tm, bx, by, bz, smem);
        else
            ok = fused_tile<S, false, false>(sb.L, (const typename S::T *)sb.f[cur], (typename S::T *)sb.f[1 - cur], sb.rho,
                                      sb.psi, sb.type, sb.zc, sb.ofs, tm, bx, by, bz, smem);
        if (!ok) break;
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
    // About 16 waves of CTAs (three per SM on 152 SMs), so the last wave's
    // idle SMs cost little, each chunk long enough (>= 16 planes where the
    // lattice allows) that its extra halo planes cost little.
    long long cols = (long long)((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY);
    int zc = L.nz;
    while (zc > 16 && cols * ((L.nz + zc - 1) / zc) < 48 * 152) zc = (zc + 1) / 2;
    return zc;
}

bool fused_plane_map(CUtensorMap *map, void *f, const Lat &L, int storage)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const size_t es = storage == LBE_STORE_F32 ? 4 : 2;
    if (!encode || ((size_t)L.nx * es) % 16 != 0) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny, (cuuint64_t)L.nz, (cuuint64_t)(2 * Q)};
    const cuuint64_t strides[3] = {(cuuint64_t)L.nx * es, (cuuint64_t)L.nx * L.ny * es, (cuuint64_t)L.S * es};
    const cuuint32_t box[4] = {TX, TY, 1, 2 * Q};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    return encode(map, dt, 4, f, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

FusedOfs fused_offsets(const Lat &L)
{
    FusedOfs ofs;
    for (int c = 0; c < 2; c++)
        for (int i = 0; i < Q; i++) {
            const long long o = (long long)(c * Q + i) * L.S, r = (long long)i * L.S;
            const long long d = cx(i) + (long long)cy(i) * L.nx + (long long)cz(i) * L.nx * L.ny;
            ofs.pop[c * Q + i] = o;
            ofs.push[c * Q + i] = o + d;
            // slot 0 never pushes; the others lie at least S - nx*ny - nx - 1 > 0
            // above the component base
            ofs.pop32[c * Q + i] = (unsigned)r;
            ofs.push32[c * Q + i] = (unsigned)(r + d);
        }
    return ofs;
}

// The 32-bit offsets hold every store of a component: the highest is slot
// 18 of the pushed neighbour plus a periodic wrap of N.
bool fused_rel32(const Lat &L)
{
    return !L.wide && (long long)Q * L.S + 2LL * L.N + (long long)L.nx * L.ny + L.nx + 1 < (1LL << 32);
}

template <class S>
static void launch_fused_t(const Lat &L, const void *fin, void *fout, const float *rho, const float *psi,
                           const uint8_t *type, const CUtensorMap *tmap, cudaStream_t s, int zc_override)
{
    static bool configured = false;  // the attribute is per function and process
    if (!configured) {
        const int b = (int)Smem<S>::bytes;
        cudaFuncSetAttribute(k_fused<S, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        cudaFuncSetAttribute(k_fused<S, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        cudaFuncSetAttribute(k_fused<S, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        cudaFuncSetAttribute(k_fused<S, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        configured = true;
    }
    const int zc = zc_override > 0 ? zc_override : fused_zchunk(L);
    dim3 grid((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY, (L.nz + zc - 1) / zc);
    FusedOfs ofs = fused_offsets(L);
    using T = typename S::T;
    const CUtensorMap none{};
    const CUtensorMap &tm = tmap ? *tmap : none;
    const bool r32 = fused_rel32(L);
    auto go = [&](auto kernel) {
        kernel<<<grid, NT, Smem<S>::bytes, s>>>(L, (const T *)fin, (T *)fout, rho, psi, type, zc, ofs, tm);
    };
    if (tmap)
        r32 ? go(k_fused<S, true, true>) : go(k_fused<S, true, false>);
    else
        r32 ? go(k_fused<S, false, true>) : go(k_fused<S, false, false>);
}

void launch_fused(int storage, const Lat &L, const void *fin, void *fout, const float *rho, const float *psi,
                  const uint8_t *type, const CUtensorMap *tmap, cudaStream_t s, int zc_override)
{
    LBE_DISPATCH(storage, (launch_fused_t<S>(L, fin, fout, rho, psi, type, tmap, s, zc_override)));
}

template <class S>
static void launch_fused_batch_t(const BatchIndex &B, int total, int ctas, cudaStream_t s)
{
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_fused_batch<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Smem<S>::bytes);
        configured = true;
    }
    k_fused_batch<S><<<ctas, NT, Smem<S>::bytes, s>>>(B, total);
}

void launch_fused_batch(int storage, const BatchIndex &B, int total_tiles, int ctas, cudaStream_t s)
{
    LBE_DISPATCH(storage, (launch_fused_batch_t<S>(B, total_tiles, ctas, s)));
}

int fused_batch_ctas_per_sm(int storage)
{
    int n = 0;
    LBE_DISPATCH(storage, (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused_batch<S>, NT, Smem<S>::bytes)));
    return n > 0 ? n : 1;
}

}  // namespace lbe
