// Fused fluid step (§2 of Günther et al., arXiv:1109.3277): densities and
// ψ = 1 - exp(-ρ) (the weight of Eq. 3), the Shan–Chen force (Eq. 3), the
// shifted-velocity BGK collision (Eq. 2) and push streaming (Eq. 1) with
// halfway bounce-back, in one pass over the populations.
//
// A CTA owns a 32 x TY column of nodes and walks a chunk of z planes.  For
// every plane of the chunk one TMA tensor copy brings the populations of
// the tile into shared memory (a box of the (x, y, z, direction) array of
// (red, blue) pairs), completing on an mbarrier.  The ψ, node type and a
// per-row bitmask of solid nodes of the tile and a one-node halo go into a
// four-slot ring of planes; the collision of plane z reads planes z-1, z
// and z+1 of it.  Two configurations fill the ring:
//  - ψ formed on chip (lattices without particles): the box also holds a
//    one-node halo (x widened to 16-byte boundaries), and each thread sums
//    the densities of its node and of at most one halo node, so ψ of the
//    tile and its halo comes from the stage; halo nodes beyond the lattice
//    edge wrap around and are read from global memory.  Solid nodes (walls)
//    take their ψ from the shell fill.
//  - ψ from memory (lattices with particles): the density pass and the
//    shell fill have written ψ of every node a fluid node sees.  The ring
//    entries of plane z + 2 arrive by asynchronous copies issued before the
//    collision of plane z and waited for after it.
//
// With τ = 1 for both components the post-collision populations are the
// equilibria, so a node's populations are needed only for its moments:
// with ψ formed on chip two stages suffice, while other τ keep three and
// re-read the node's populations at the collision.  With ψ from memory a
// third stage (copies two planes ahead) is kept where it costs no CTA per
// SM.
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

constexpr int TX = FUSED_TX;

__device__ __forceinline__ int wrapc(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Compile-time layout of one configuration: storage S, tile rows TY, GEN
// (any τ) or not (τ = 1), and SELF (the box holds
// the tile and a one-node halo, whose densities the kernel forms itself) or
// not (the box holds the tile; ψ of every ring entry comes from memory).
template <class S, int TY, bool GEN, bool SELF>
struct Cfg {
    using P = typename S::P;
    static constexpr int NT = TX * TY;
    static constexpr int E = (int)sizeof(P);          // bytes of one (red, blue) pair
    static constexpr int PADX = SELF ? 16 / E : 0;    // x margin of the box: 16 bytes
    static constexpr int BX = TX + 2 * PADX, BY = SELF ? TY + 2 : TY;
    static constexpr int HX = TX + 2, HY = TY + 2, HN = HX * HY, NHALO = HN - NT;
    static constexpr size_t plane = (size_t)Q * BY * BX * E;        // bytes of one box
    static constexpr size_t pstride = (plane + 127) / 128 * 128;    // stages 128-byte aligned
    // CTAs per SM the kernel is compiled for: what shared memory allows
    // (228 KB per SM, about 1 KB of it reserved per CTA), capped so that a
    // thread keeps at least 80 registers (τ = 1: 768 threads per SM) or 128
    // (any τ: 512), which the node arithmetic needs without spilling.
    static constexpr int by_regs = (GEN ? 512 : 768) / NT;
    static constexpr size_t twords = SELF ? 0 : (size_t)NT * 4 * sizeof(uint32_t);  // type words in flight
    static constexpr size_t other =
        4 * HN * sizeof(float2) + 4 * HY * sizeof(unsigned long long) + twords + 128 + 1024;
    static constexpr int ctas_for(int nst)
    {
        const int m = (int)((228 * 1024) / (nst * pstride + nst * 8 + other));
        return m < by_regs ? (m > 0 ? m : 1) : by_regs;
    }
    // stage buffers: any τ with SELF re-reads plane z's box one iteration
    // after its densities (three); otherwise a box is done with in the
    // iteration it arrives, and a third buffer lets the copies run two
    // planes ahead where it costs no CTA per SM
    static constexpr int NST = (GEN && SELF) ? 3 : (SELF ? 2 : (ctas_for(3) >= ctas_for(2) ? 3 : 2));
    static constexpr int CTAS = ctas_for(NST);
    // dynamic shared memory (bytes from a 128-byte aligned base)
    static constexpr size_t stage = 0;                              // P [NST][Q][BY][BX]
    static constexpr size_t sps = stage + NST * pstride;            // float2 [4][HN] (ψ_b, ψ_r)
    static constexpr size_t smask = sps + 4 * HN * sizeof(float2);  // uint64 [4][HY] solid bits per row
    static constexpr size_t stw = smask + 4 * HY * sizeof(unsigned long long);  // uint32 [NT][4] type words
    static constexpr size_t bar = stw + twords;                     // uint64 [NST] mbarriers
    static constexpr size_t bytes = bar + NST * sizeof(unsigned long long) + 128;  // + alignment slack
};

// Per stage buffer counters kept in registers (every index a compile-time
// constant after unrolling).
template <int N>
struct Counts {
    int v[N];
    __device__ __forceinline__ int get(int b) const
    {
        int r = v[0];
#pragma unroll
        for (int j = 1; j < N; j++)
            if (b == j) r = v[j];
        return r;
    }
    __device__ __forceinline__ void inc(int b)
    {
#pragma unroll
        for (int j = 0; j < N; j++)
            if (b == j) v[j]++;
    }
};

// The first 128-byte aligned byte at or after p.  The result is a generic
// address (rounded through an integer), so the compiler issues generic
// loads for the box, ring and mask reads: measured faster for this kernel
// than shared-memory instructions, which stall on their issue queue.
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

// order earlier shared-memory accesses before later TMA writes
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

// Non-blocking look at the phase with this parity.
__device__ __forceinline__ bool mbar_test_wait(unsigned long long *b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with this parity; false if it has not completed
// within `limit` tries: a non-blocking look, then tries that may each
// suspend the thread for a while.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, unsigned parity, int limit)
{
    if (mbar_test_wait(b, parity)) return true;
    for (int k = 1; k < limit; k++)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

// One box of the 4D tensor of population pairs (x, y, z, direction) at
// (x0, y0, z, 0) into shared memory, completing on b.  x0 * pair bytes is a
// multiple of 16 (x0 = tile start - 16 bytes); out-of-range elements
// (x0 or y0 negative, past the lattice) are filled with zeros.
__device__ __forceinline__ void tma_box(void *dst, const CUtensorMap *map, int x0, int y0, int z,
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
//
// The two components go through the same node arithmetic, so it is done on
// (red, blue) pairs with the paired FP32 instructions (add, subtract,
// multiply and fused multiply-add on two lanes, each rounded to nearest
// like its scalar form; the subtraction, which has no intrinsic, in PTX):
// every component's result has the bits of the scalar sequence.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{\n"
        " .reg .b64 ra, rb, rd;\n"
        " mov.b64 ra, {%2, %3};\n"
        " mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n"
        " mov.b64 {%0, %1}, rd;\n"
        "}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
struct Add2 {
    __device__ __forceinline__ float2 operator()(float2 a, float2 b) const { return add2(a, b); }
};

// Reciprocal by the hardware approximation (PTX rcp.approx; error of the
// order of one unit in the last place): the inverse densities of the
// equilibrium velocity.  Like the other operations it gives the same bits
// wherever it is inlined.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Σ_k c_{2k+1} d_k over the nine opposite pairs (2k+1, 2k+2), where d_k is
// the quantity of direction 2k+1 minus that of 2k+2 (c_{2k+2} = -c_{2k+1}):
// the three Cartesian components, terms added in k order as they come.
// c_1, c_3, c_5 are the unit vectors x, y, z: each component starts there.
__device__ __forceinline__ void odd_put(float2 out[3], int k, float2 d)
{
    const int i = 2 * k + 1;
    const int c[3] = {cx(i), cy(i), cz(i)};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (!c[a]) continue;
        if (k == a)
            out[a] = d;
        else
            out[a] = c[a] > 0 ? add2(out[a], d) : sub2(out[a], d);
    }
}

// Moments of the stored quantities d_i (δf_i at 16 bit, f_i in FP32) of a
// node: Δρ^c = Σ_i d_i (in the order of PairTree) and j^c = Σ_i c_i
// d_i (the bases w_i ρ_ref cancel in j, since Σ_i w_i c_i = 0).  ld(i)
// gives the (red, blue) pair of direction i.
struct Mom {
    float2 dr;     // Δρ = ρ - ρ_ref (ρ itself in FP32)
    float2 j[3];
};

template <class LD>
__device__ __forceinline__ Mom moments(LD ld)
{
    Mom m;
    PairTree t;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const float2 va = ld(2 * k + 1), vb = ld(2 * k + 2);
        t.put(k, add2(va, vb), Add2{});
        odd_put(m.j, k, sub2(va, vb));
    }
    m.dr = t.finish(ld(0), Add2{});
    return m;
}

// Σ_i d_i alone (a halo node needs its density only), in the same order.
template <class LD>
__device__ __forceinline__ float2 density_sum(LD ld)
{
    PairTree t;
#pragma unroll
    for (int k = 0; k < 9; k++) t.put(k, add2(ld(2 * k + 1), ld(2 * k + 2)), Add2{});
    return t.finish(ld(0), Add2{});
}

// Equilibrium velocities of both components, u' + (τ_c/ρ_c) F^c with the
// Shan–Chen force F^c = -g ψ^c s^c + ρ^c g_body (Eq. 3), and -1.5 u·u.
// TAU1 (τ = 1 for both) skips the products with τ_c = 1, which are exact:
// the same bits as the general form.
template <bool TAU1>
__device__ __forceinline__ void eq_velocity(const Lat &L, float2 r, float2 pc, const float2 s[3], const float up[3],
                                            float2 ue[3], float2 &um15)
{
    float2 ir = make_float2(r.x > 0.f ? rcp_approx(r.x) : 0.f, r.y > 0.f ? rcp_approx(r.y) : 0.f);
    if (!TAU1) ir = mul2(make_float2(L.tau[0], L.tau[1]), ir);
    const float2 gp = mul2(dup2(-L.g), pc);
    if (L.body[0] != 0.f || L.body[1] != 0.f || L.body[2] != 0.f) {
#pragma unroll
        for (int k = 0; k < 3; k++) ue[k] = fma2(ir, fma2(gp, s[k], mul2(r, dup2(L.body[k]))), dup2(up[k]));
    } else {
#pragma unroll
        for (int k = 0; k < 3; k++) ue[k] = fma2(ir, mul2(gp, s[k]), dup2(up[k]));
    }
    const float2 uu = fma2(ue[0], ue[0], fma2(ue[1], ue[1], mul2(ue[2], ue[2])));
    um15 = mul2(dup2(-1.5f), uu);
}

// c_i·u for odd i: the first non-zero component of c_i is +1, the second
// (diagonals) ±1.
__device__ __forceinline__ float2 cu_odd(int i, const float2 ue[3])
{
    const int c[3] = {cx(i), cy(i), cz(i)};
    float2 r = dup2(0.f);
    bool first = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (!c[a]) continue;
        r = first ? ue[a] : (c[a] > 0 ? add2(r, ue[a]) : sub2(r, ue[a]));
        first = false;
    }
    return r;
}

// BGK relaxation f + (f^eq - f)/τ; a component with τ = 1 takes f^eq
// itself, the value the τ = 1 kernels store without reading f.
__device__ __forceinline__ float2 relax(float2 f, float2 feq, float2 it)
{
    const float2 r = fma2(sub2(feq, f), it, f);
    return make_float2(it.x == 1.f ? feq.x : r.x, it.y == 1.f ? feq.y : r.y);
}

// Halo entry h of the (32 + 2) x (TY + 2) ring: top row, bottom row, left
// column, right column.
template <int TY>
__device__ __forceinline__ void halo_entry(int h, int &ex, int &ey)
{
    constexpr int HX = TX + 2, HY = TY + 2;
    if (h < HX) {
        ex = h;
        ey = 0;
    } else if (h < 2 * HX) {
        ex = h - HX;
        ey = HY - 1;
    } else if (h < 2 * HX + TY) {
        ex = 0;
        ey = h - 2 * HX + 1;
    } else {
        ex = HX - 1;
        ey = h - 2 * HX - TY + 1;
    }
}

// A ring entry a thread looks after: its place in the ring and in a staged
// box, its wrapped lattice column (x + nx y), and whether the box holds it
// (otherwise it is read from global memory).
struct Ent {
    int ring, st, xy, ex, ey;
    bool inlat;
};

constexpr int WAIT_LIMIT = FUSED_WAIT_LIMIT;

// One tile (column bx, by, z chunk bz) of one lattice.  TMA: the boxes
// arrive as tensor copies described by *tmap; otherwise every entry is read
// from global memory.  Each wait for a box tries wait_limit times; if one
// runs out the CTA stops, waits (with the full limit) for its copies in
// flight, records the timeout in the lattice's status word and returns
// false.  A negative wait_limit makes every wait one that nothing completes
// (tests).  SELF: ψ of fluid nodes is formed here from the densities of the
// box; otherwise psi holds ψ of every node (the density kernel's and the
// shell fill's), and the box holds the tile only.
template <class S, int TY, bool GEN, bool SELF, bool TMA, bool R32>
__device__ __forceinline__ bool fused_tile(const Lat &L, const typename S::P *__restrict__ fin,
                                           typename S::P *__restrict__ fout, const float *__restrict__ psi,
                                           const uint8_t *__restrict__ type, int zc, const FusedOfs &ofs,
                                           const CUtensorMap *tmap, int bx, int by, int bz, int wait_limit,
                                           unsigned char *smem)
{
    using C = Cfg<S, TY, GEN, SELF>;
    using P = typename S::P;
    constexpr int HX = C::HX, HN = C::HN, BX = C::BX, BY = C::BY, NST = C::NST;
    constexpr size_t PSTR = C::pstride / sizeof(P);  // pairs from one stage to the next
    const P *stage = reinterpret_cast<const P *>(smem + C::stage);
    float2 *sps = reinterpret_cast<float2 *>(smem + C::sps);                                // [slot][e]
    unsigned long long *smask = reinterpret_cast<unsigned long long *>(smem + C::smask);   // [slot][ey]
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem + C::bar);
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int x0 = bx * TX, y0 = by * TY;
    const int zb = bz * zc, ze = min(zb + zc, L.nz);
    // wait_limit < 0 (tests of the timeout path): every wait for a box is
    // for the barrier's next phase, which no copy completes, with |limit|
    // tries; the cleanup below still waits for the copies in flight
    const unsigned unreachable = wait_limit < 0 ? 1u : 0u;
    const int limit = wait_limit < 0 ? -wait_limit : wait_limit;
    const int nxy = L.nx * L.ny;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < L.nx && gy < L.ny;

    auto make_ent = [&](int ex, int ey) {
        Ent e;
        e.ex = ex;
        e.ey = ey;
        e.ring = ey * HX + ex;
        const int lx = x0 - 1 + ex, ly = y0 - 1 + ey;
        if (SELF) {
            e.st = ey * BX + ex - 1 + C::PADX;
            e.inlat = TMA && lx >= 0 && lx < L.nx && ly >= 0 && ly < L.ny;
        } else {  // only the own entries of active nodes are in the box
            e.st = (ey - 1) * BX + ex - 1;
            e.inlat = TMA && ex >= 1 && ex <= TX && ey >= 1 && ey <= TY && lx < L.nx && ly < L.ny;
        }
        e.xy = wrapc(lx, L.nx) + L.nx * wrapc(ly, L.ny);
        return e;
    };
    const Ent own = make_ent(tx + 1, ty + 1);
    const bool has_halo = tid < C::NHALO;
    Ent hal{};
    if (has_halo) {
        int ex, ey;
        halo_entry<TY>(tid, ex, ey);
        hal = make_ent(ex, ey);
    }

    // iteration k handles ring plane zb - 1 + k: its box arrives, its
    // entries go into ring slot k & 3, and plane zb - 2 + k (k >= 2) is
    // collided
    const int kmax = ze - zb + 2;
    auto pvalid = [&](int p) { return !L.walls || (p >= 0 && p < L.nz); };
    auto gz_of = [&](int p) { return p < 0 ? p + L.nz : (p >= L.nz ? p - L.nz : p); };  // p in [-1, nz]
    // per stage buffer: boxes issued (thread 0) and waited for (every thread)
    Counts<NST> issued{}, waited{};
    auto issue = [&](int k, int b) {
        if (!TMA || tid != 0) return;
        const int p = zb - 1 + k;
        if (!pvalid(p)) return;
        fence_proxy_async();
        mbar_expect_tx(&bar[b], (unsigned)C::plane);
        tma_box(const_cast<P *>(stage) + (size_t)b * PSTR, tmap, x0 - C::PADX, y0 - (SELF ? 1 : 0), gz_of(p),
                &bar[b]);
        issued.inc(b);
    };

    // node types one plane ahead, and ψ: SELF loads it for solid nodes
    // only (once their type is known), otherwise for every node along
    // with the type
    auto load_type = [&](int k, const Ent &e) -> uint8_t {
        const int p = zb - 1 + k;
        if (!pvalid(p)) return WALL;
        return type[e.xy + (size_t)nxy * gz_of(p)];
    };
    auto load_psi = [&](int k, const Ent &e, uint8_t t) -> float2 {
        const int p = zb - 1 + k;
        if ((SELF && t == FLUID) || !pvalid(p)) return dup2(0.f);
        const size_t n = e.xy + (size_t)nxy * gz_of(p);
        return make_float2(psi[n], psi[(size_t)L.N + n]);
    };

    // Collision of plane z with ring slots s0, s1, s2 (planes z - 1, z,
    // z + 1): the own node's moments from mom_of(), with GEN its stored
    // pairs from stage buffer bst (or global memory) for the relaxation.
    auto collide_at = [&](int z, int s0, int s1, int s2, int bst, auto mom_of) {
        const float2 *pl[3] = {sps + s0 * HN, sps + s1 * HN, sps + s2 * HN};
        const unsigned long long *ml[3] = {smask + s0 * C::HY, smask + s1 * C::HY, smask + s2 * C::HY};
        const bool solid_own = (ml[1][ty + 1] >> (tx + 1)) & 1ull;
        const int n = gx + L.nx * gy + nxy * z;
        if (active && !solid_own) {
            const Mom mcur = mom_of();
            const float2 rref2 = make_float2(L.rref[0], L.rref[1]);
            const float2 drho = mcur.dr, rho_ = add2(rref2, mcur.dr);
            // u' = Σ_c j^c/τ_c / Σ_c ρ^c/τ_c; with τ = 1 the products with
            // 1/τ_c = 1 are exact and left out (the same bits)
            const float den = GEN ? __fmaf_rn(rho_.y, L.itau[1], __fmul_rn(rho_.x, L.itau[0]))
                                  : __fadd_rn(rho_.x, rho_.y);
            const float iden = den > 0.f ? rcp_approx(den) : 0.f;
            float up[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const float jt = GEN ? __fmaf_rn(mcur.j[d].y, L.itau[1], __fmul_rn(mcur.j[d].x, L.itau[0]))
                                     : __fadd_rn(mcur.j[d].x, mcur.j[d].y);
                up[d] = __fmul_rn(jt, iden);
            }
            // s^c = Σ_i c_i ψ^{c'}(x + c_i) over opposite pairs: the ring
            // holds (ψ_b, ψ_r), the partner of (red, blue)
            float2 s[3];
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const int i = 2 * k + 1;
                odd_put(s, k, sub2(pl[cz(i) + 1][own.ring + cy(i) * HX + cx(i)],
                                   pl[1 - cz(i)][own.ring - cy(i) * HX - cx(i)]));
            }
            const float2 pcc = pl[1][own.ring];
            const float2 pc = make_float2(pcc.y, pcc.x);  // own (ψ_r, ψ_b)
            // solid rows around this warp's row (the same for all its
            // lanes) and whether its nodes lie on a periodic boundary:
            // mode 0 (neither, all nodes active) pushes every population to
            // its fixed offset; mode 1 (solid neighbours) reflects where
            // the neighbour is solid; mode 2 also wraps the push offsets
            unsigned long long mrow = 0ull;
#pragma unroll
            for (int dz = 0; dz < 3; dz++)
#pragma unroll
                for (int dy = 0; dy < 3; dy++) mrow |= ml[dz][ty + dy];
            const bool inner_x = x0 > 0 && x0 + TX < L.nx;
            const bool inner_y = gy > 0 && gy < L.ny - 1;
            const bool inner_z = L.walls || (z > 0 && z < L.nz - 1);
            const bool inner = inner_x && inner_y && inner_z;
            P *dst = fout + n;
            auto collide = [&](auto mode_tag) {
                constexpr int MODE = decltype(mode_tag)::value;
                // bit (cx+1) + 3 (cy+1) + 9 (cz+1): neighbour is solid
                uint32_t nb27 = 0;
                int wx[2] = {0, 0}, wy[2] = {0, 0}, wz[2] = {0, 0};
                if (MODE >= 1) {
#pragma unroll
                    for (int dz = 0; dz < 3; dz++)
#pragma unroll
                        for (int dy = 0; dy < 3; dy++) {
                            const unsigned long long m = ml[dz][ty + dy];
                            const uint32_t f3 =
                                __funnelshift_r((uint32_t)m, (uint32_t)(m >> 32), (uint32_t)tx) & 7u;
                            nb27 |= f3 << (3 * (dy + 3 * dz));
                        }
                }
                if (MODE == 2) {
                    // push offsets of nodes on the lattice boundary wrap
                    // around the periodic axes: corrections for c = +1
                    // ([0]) and c = -1 ([1])
                    wx[0] = gx == L.nx - 1 ? -L.nx : 0;
                    wx[1] = gx == 0 ? L.nx : 0;
                    wy[0] = gy == L.ny - 1 ? -nxy : 0;
                    wy[1] = gy == 0 ? nxy : 0;
                    if (!L.walls) {  // with walls z = 0 and nz-1 are wall nodes
                        wz[0] = z == L.nz - 1 ? -L.N : 0;
                        wz[1] = z == 0 ? L.N : 0;
                    }
                }
                // store of the post-collision pair of direction i: pushed
                // to the neighbour, or reflected into slot opp(i) of this
                // node (walls and particle nodes; the link kernel adds
                // the moving-boundary term for the latter).  Both slots
                // have the same weight, hence the same storage offset;
                // the address is a select, not a branch.
                auto put = [&](int i, float2 fs) {
                    const P v = S::enc2(fs);
                    if (MODE == 0) {
                        if constexpr (R32)
                            dst[ofs.push32[i]] = v;
                        else
                            dst[ofs.push[i]] = v;
                    } else {
                        const int bit = (cx(i) + 1) + 3 * ((cy(i) + 1) + 3 * (cz(i) + 1));
                        const bool sol = (nb27 >> bit) & 1u;
                        const int corr = (cx(i) > 0 ? wx[0] : (cx(i) < 0 ? wx[1] : 0)) +
                                         (cy(i) > 0 ? wy[0] : (cy(i) < 0 ? wy[1] : 0)) +
                                         (cz(i) > 0 ? wz[0] : (cz(i) < 0 ? wz[1] : 0));
                        if constexpr (R32) {
                            const unsigned o = sol ? ofs.pop32[opp(i)] : ofs.push32[i] + (unsigned)corr;
                            dst[o] = v;
                        } else {
                            const long long o = sol ? ofs.pop[opp(i)] : ofs.push[i] + corr;
                            dst[o] = v;
                        }
                    }
                };
                // GEN: the node's stored pairs for the relaxation, from
                // the box of plane z (or global memory)
                const P *fb = stage + (size_t)bst * PSTR + own.st;
                auto ldf = [&](int i) {
                    if (TMA) return S::raw2(fb[i * BY * BX]);
                    return S::raw2(fin[pidx(L, i, (long long)n)]);
                };
                float2 ue[3], um15;
                eq_velocity<!GEN>(L, rho_, pc, s, up, ue, um15);
                const float2 it = make_float2(L.itau[0], L.itau[1]);
                // f^eq_i relative to the stored quantity's base w_i ρ_ref:
                // w_i (ρ (4.5 (c·u)^2 - 1.5 u·u) + Δρ) ± 3 w_i ρ c·u for the
                // opposite pair (i, i+1), with per weight (axis 1/18,
                // diagonal 1/36) A = w (ρ (-1.5 u·u) + Δρ), B = 4.5 w ρ and
                // C = 3 w ρ (Δρ = ρ, base 0 in FP32)
                const float2 a0 = fma2(rho_, um15, drho);
                const float2 A[2] = {mul2(dup2(wgt(1)), a0), mul2(dup2(wgt(7)), a0)};
                const float2 B[2] = {mul2(dup2(4.5f * wgt(1)), rho_), mul2(dup2(4.5f * wgt(7)), rho_)};
                const float2 Cp[2] = {mul2(dup2(3.f * wgt(1)), rho_), mul2(dup2(3.f * wgt(7)), rho_)};
                const float2 Cm[2] = {mul2(dup2(-3.f * wgt(1)), rho_), mul2(dup2(-3.f * wgt(7)), rho_)};
                float2 seq[2];  // Σ of the even parts per weight
#pragma unroll
                for (int i = 1; i < Q; i += 2) {
                    const int wc = i < 7 ? 0 : 1;
                    const float2 cu = cu_odd(i, ue);
                    const float2 even = fma2(mul2(B[wc], cu), cu, A[wc]);
                    seq[wc] = i == 1 || i == 7 ? even : add2(seq[wc], even);
                    float2 ra = fma2(Cp[wc], cu, even), rb = fma2(Cm[wc], cu, even);
                    if (GEN) {
                        ra = relax(ldf(i), ra, it);
                        rb = relax(ldf(i + 1), rb, it);
                    }
                    put(i, ra);
                    put(i + 1, rb);
                }
                // rest population: Δρ - Σ_{i>0} f^eq_i in the stored
                // quantity, so that the equilibria carry the node's mass
                float2 r0 = fma2(dup2(-2.f), add2(seq[0], seq[1]), drho);
                if (GEN) r0 = relax(ldf(0), r0, it);
                dst[0] = S::enc2(r0);
            };
            if (inner && mrow == 0ull)
                collide(std::integral_constant<int, 0>{});
            else if (inner)
                collide(std::integral_constant<int, 1>{});
            else
                collide(std::integral_constant<int, 2>{});
        } else if (active) {
            // A solid node's populations are never read (a node that a
            // particle uncovers gets f^eq in all slots), but writing them
            // keeps every sector of the output fully written: a partly
            // written sector costs a DRAM read when it leaves L2.
            P *d0 = fout + n;
            const P zero = S::enc2(make_float2(0.f, 0.f));
#pragma unroll
            for (int i = 0; i < Q; i++) {
                if constexpr (R32)
                    d0[ofs.pop32[i]] = zero;
                else
                    d0[ofs.pop[i]] = zero;
            }
        }
    };

    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < NST; b++) mbar_init(&bar[b], 1);
        fence_barrier_init();
    }
    bool ok = true;
    if constexpr (!SELF) {
        // Without SELF the ring runs two planes ahead of the collision: the
        // entries of plane z + 2 are copied into their ring slot (which the
        // collision of plane z does not read) by asynchronous copies issued
        // before the collision and waited for after it, so that their
        // latency is hidden behind it: ψ straight into the slot, the 32-bit
        // word holding each entry's node type into per-thread scratch.  Each
        // warp puts whole ring rows (its own row, with the side entries
        // taken by lanes 30 and 31; warps 0 and 1 also the halo rows 0 and
        // TY + 1, two entries for lanes 0 and 1), so after the wait it forms
        // their solid bits with ballots and one lane writes each row's word:
        // one barrier per plane, at its end, which also makes the copies
        // visible and gathers the copy timeouts.  The own node's moments
        // come from the box of plane z at the collision.
        const int lane = tx, warp = ty;
        const bool has_a = warp < 2, has_b = warp < 2 && lane < 2, has_c = lane >= 30;
        const int hrow = warp == 0 ? 0 : TY + 1;
        const Ent ha = make_ent(lane, hrow), hb = make_ent(lane + 32, hrow);
        const Ent hc = make_ent(lane == 30 ? 0 : HX - 1, warp + 1);
        uint32_t *tw = reinterpret_cast<uint32_t *>(smem + C::stw) + 4 * tid;  // own, a, b, c
        auto cp4 = [](void *dst, const void *src) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
        };
        auto ring_fetch = [&](int k, int slot) {
            const int p = zb - 1 + k;
            const bool pv = pvalid(p);
            const size_t g = pv ? (size_t)nxy * gz_of(p) : 0;
            float2 *ps = sps + slot * HN;
            auto one = [&](const Ent &e, int q) {
                float2 *d = ps + e.ring;
                if (!pv) {  // beyond a wall: solid, ψ = 0
                    *d = dup2(0.f);
                    tw[q] = 0x01010101u * WALL;
                    return;
                }
                const size_t n = e.xy + g;
                cp4(&d->x, psi + (size_t)L.N + n);  // (ψ_b, ψ_r): the partner first
                cp4(&d->y, psi + n);
                cp4(&tw[q], reinterpret_cast<const void *>(reinterpret_cast<uintptr_t>(type + n) & ~uintptr_t(3)));
            };
            one(own, 0);
            if (has_a) one(ha, 1);
            if (has_b) one(hb, 2);
            if (has_c) one(hc, 3);
        };
        auto ring_masks = [&](int k, int slot) {
            asm volatile("cp.async.wait_all;" ::: "memory");
            const int p = zb - 1 + k;
            const size_t g = pvalid(p) ? (size_t)nxy * gz_of(p) : 0;
            auto solid = [&](const Ent &e, int q) {
                const unsigned sh = 8u * (unsigned)(reinterpret_cast<uintptr_t>(type + e.xy + g) & 3u);
                return ((tw[q] >> sh) & 0xFFu) != FLUID;
            };
            const unsigned bo = __ballot_sync(0xffffffffu, solid(own, 0));
            const unsigned ba = __ballot_sync(0xffffffffu, has_a && solid(ha, 1));
            const unsigned bb = __ballot_sync(0xffffffffu, has_b && solid(hb, 2));
            const unsigned bc = __ballot_sync(0xffffffffu, has_c && solid(hc, 3));
            if (lane == 0) {
                smask[slot * C::HY + warp + 1] = ((unsigned long long)bo << 1) | ((bc >> 30) & 1u) |
                                                 ((unsigned long long)((bc >> 31) & 1u) << 33);
                if (has_a)
                    smask[slot * C::HY + hrow] = (unsigned long long)ba | ((unsigned long long)(bb & 3u) << 32);
            }
        };
        auto issue_z = [&](int z, int b) {
            if (!TMA || tid != 0) return;
            fence_proxy_async();
            mbar_expect_tx(&bar[b], (unsigned)C::plane);
            tma_box(const_cast<P *>(stage) + (size_t)b * PSTR, tmap, x0, y0, z, &bar[b]);
            issued.inc(b);
        };
        __syncthreads();  // barriers initialised
        // plane zb + j arrives in stage buffer j mod NST; the copies run
        // NST - 1 planes ahead
#pragma unroll
        for (int q = 0; q + 1 < NST; q++)
            if (zb + q < ze) issue_z(zb + q, q);
        // ring planes zb - 1, zb, zb + 1 (index k = plane - zb + 1)
        for (int k = 0; k < 3; k++) {
            ring_fetch(k, k);
            ring_masks(k, k);
        }
        __syncthreads();
        int b = 0;
        for (int j = 0; j < ze - zb; j++) {
            const int z = zb + j;
            const int b_ahead = b == 0 ? NST - 1 : b - 1;  // (j + NST - 1) mod NST
            if (z + NST - 1 < ze) issue_z(z + NST - 1, b_ahead);
            const int kn = j + 3;  // ring index of plane z + 2
            if (kn < kmax) ring_fetch(kn, kn & 3);
            bool late = false;
            if (TMA) {
                late = !mbar_wait(&bar[b], (unsigned)(waited.get(b) & 1) ^ unreachable, limit);
                if (!late) waited.inc(b);
            }
            // a copy that never arrived leaves stale shared data: the
            // collision then stores garbage (at valid addresses), and the
            // step is reported as timed out
            collide_at(z, j & 3, (j + 1) & 3, (j + 2) & 3, b, [&] {
                const P *sb = stage + (size_t)b * PSTR;
                if (TMA) return moments([&](int i) { return S::raw2(sb[i * BY * BX + own.st]); });
                const size_t n = own.xy + (size_t)nxy * z;
                return moments([&](int i) { return S::raw2(fin[pidx(L, i, (long long)n)]); });
            });
            if (kn < kmax) ring_masks(kn, kn & 3);
            b = b + 1 == NST ? 0 : b + 1;
            if (__syncthreads_or(late)) {
                ok = false;
                break;
            }
        }
    } else {
        if (tid < C::HY) smask[tid] = 0ull;  // slot 0
        __syncthreads();
        issue(0, 0);
        uint8_t t_own = load_type(0, own), t_hal = has_halo ? load_type(0, hal) : WALL;
        float2 p_own = load_psi(0, own, t_own), p_hal = has_halo ? load_psi(0, hal, t_hal) : dup2(0.f);
        Mom mcur{}, mnext{};
            int b_cur = 0;  // stage buffer of iteration k
        for (int k = 0; k < kmax; k++) {
            const int b_next = b_cur + 1 == NST ? 0 : b_cur + 1;
            const int b_prev = b_cur == 0 ? NST - 1 : b_cur - 1;
            if (k + 1 < kmax) issue(k + 1, b_next);
            const int p = zb - 1 + k;
            const bool pv = pvalid(p);
            // types (and without SELF ψ) of the next plane: in flight during this iteration
            uint8_t tn_own = WALL, tn_hal = WALL;
            float2 pn_own = dup2(0.f), pn_hal = dup2(0.f);
            if (k + 1 < kmax) {
                tn_own = load_type(k + 1, own);
                if (has_halo) tn_hal = load_type(k + 1, hal);
                if (!SELF) {
                    pn_own = load_psi(k + 1, own, tn_own);
                    if (has_halo) pn_hal = load_psi(k + 1, hal, tn_hal);
                }
            }
            bool late = false;
            if (TMA && pv) {
                late = !mbar_wait(&bar[b_cur], (unsigned)(waited.get(b_cur) & 1) ^ unreachable, limit);
                if (!late) waited.inc(b_cur);
            }
            if (__syncthreads_or(late)) {
                ok = false;
                break;
            }
            // this plane's entries into ring slot k & 3: ψ (formed here for
            // fluid nodes with SELF), type, solid bits; the own node's moments
            {
                const int slot = k & 3;
                const P *sb = stage + (size_t)b_cur * PSTR;
                const size_t gbase = pv ? (size_t)nxy * gz_of(p) : 0;
                auto entry = [&](const Ent &e, uint8_t t, float2 ps, bool is_own) {
                    float2 pq = ps;  // (ψ_r, ψ_b)
                    if (t == FLUID && pv && (SELF || is_own)) {
                        float2 dr;
                        if (e.inlat) {
                            auto ld = [&](int i) { return S::raw2(sb[i * BY * BX + e.st]); };
                            if (is_own) {
                                mnext = moments(ld);
                                dr = mnext.dr;
                            } else {
                                dr = density_sum(ld);
                            }
                        } else {
                            const size_t n = e.xy + gbase;
                            auto ld = [&](int i) { return S::raw2(fin[pidx(L, i, (long long)n)]); };
                            if (is_own) {
                                mnext = moments(ld);
                                dr = mnext.dr;
                            } else {
                                dr = density_sum(ld);
                            }
                        }
                        if (SELF) {
                            const float2 r = add2(make_float2(L.rref[0], L.rref[1]), dr);
                            pq = make_float2(1.f - expf(-r.x), 1.f - expf(-r.y));
                        }
                    }
                    sps[slot * HN + e.ring] = make_float2(pq.y, pq.x);  // (ψ_b, ψ_r): the partner first
                    if (t != FLUID) atomicOr(&smask[slot * C::HY + e.ey], 1ull << e.ex);
                };
                // without SELF an own entry of an inactive node holds no moments
                entry(own, t_own, p_own, SELF || active);
                if (has_halo) entry(hal, t_hal, p_hal, false);
            }
            __syncthreads();
            // collision of plane z = p - 1 with ring planes z - 1, z, z + 1
            if (k >= 2) collide_at(p - 1, (k - 2) & 3, (k - 1) & 3, k & 3, b_prev, [&] { return mcur; });
            mcur = mnext;
            // ring slot (k+1) & 3 was last read by the collision of iteration
            // k - 1: clear its solid rows for the next iteration
            if (tid < C::HY) smask[((k + 1) & 3) * C::HY + tid] = 0ull;
            // SELF: ψ of the next plane's solid entries, now that their types are in
            t_own = tn_own;
            t_hal = tn_hal;
            if (SELF && k + 1 < kmax) {
                p_own = load_psi(k + 1, own, t_own);
                if (has_halo) p_hal = load_psi(k + 1, hal, t_hal);
            } else {
                p_own = pn_own;
                p_hal = pn_hal;
            }
            b_cur = b_next;
            __syncthreads();
        }
    }
    if (TMA) {
        if (tid == 0) {
            // let the copies in flight land (bounded) before the memory is reused
            bool lost = !ok;
#pragma unroll
            for (int b = 0; b < NST; b++)
                for (int u = waited.get(b); u < issued.get(b); u++)
                    if (!mbar_wait(&bar[b], (unsigned)(u & 1), WAIT_LIMIT)) lost = true;
            if (lost) atomicOr(L.status, 1u);
        }
        __syncthreads();
        if (tid == 0)
#pragma unroll
            for (int b = 0; b < NST; b++) mbar_inval(&bar[b]);
    }
    return ok;
}

template <class S, int TY, bool GEN, bool SELF, bool TMA, bool R32>
__global__ void __launch_bounds__(TX *TY, (Cfg<S, TY, GEN, SELF>::CTAS))
    k_fused(Lat L, const typename S::P *__restrict__ fin, typename S::P *__restrict__ fout,
            const float *__restrict__ psi, const uint8_t *__restrict__ type, int zc, FusedOfs ofs,
            const __grid_constant__ CUtensorMap tmap, int wait_limit)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    fused_tile<S, TY, GEN, SELF, TMA, R32>(L, fin, fout, psi, type, zc, ofs, &tmap, blockIdx.x, blockIdx.y,
                                           blockIdx.z, wait_limit, align128(smem_raw));
}

// Persistent multi-lattice variant: CTAs take tiles of all boxes of a batch
// from one queue (largest boxes first in the queue order set by the host).
// It runs the any-τ configuration with ψ from memory (the batch runs the
// density kernel), which stores exactly what the other configurations
// store: τ = 1 takes f^eq in the relaxation, and ψ from memory has the
// bits of ψ formed in the kernel.
constexpr int BATCH_TY = FUSED_TY_BATCH;

template <class S>
__global__ void __launch_bounds__(TX *BATCH_TY, (Cfg<S, BATCH_TY, true, false>::CTAS)) k_fused_batch(BatchIndex B, int total)
{
    constexpr int NT = TX * BATCH_TY;
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
        using P = typename S::P;
        bool ok;
        if (sb.tma)
            ok = fused_tile<S, BATCH_TY, true, false, true, false>(sb.L, (const P *)sb.f[cur], (P *)sb.f[1 - cur], sb.psi,
                                                            sb.type, sb.zc, sb.ofs, tm, bx, by, bz, WAIT_LIMIT, smem);
        else
            ok = fused_tile<S, BATCH_TY, true, false, false, false>(sb.L, (const P *)sb.f[cur], (P *)sb.f[1 - cur], sb.psi,
                                                             sb.type, sb.zc, sb.ofs, tm, bx, by, bz, WAIT_LIMIT, smem);
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

int fused_zchunk(const Lat &L, int ty)
{
    // About 16 waves of CTAs (three per SM on 152 SMs), so the last wave's
    // idle SMs cost little, each chunk long enough (>= 16 planes where the
    // lattice allows) that its two extra halo planes cost little.
    long long cols = (long long)((L.nx + TX - 1) / TX) * ((L.ny + ty - 1) / ty);
    int zc = L.nz;
    while (zc > 16 && cols * ((L.nz + zc - 1) / zc) < 48 * 152) zc = (zc + 1) / 2;
    return zc;
}

bool fused_tau1(const Lat &L) { return L.itau[0] == 1.f && L.itau[1] == 1.f; }

bool fused_plane_map(CUtensorMap *map, void *f, const Lat &L, int storage, int ty, bool self)
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
    // one element = the (red, blue) pair of a population
    const size_t es = storage == LBE_STORE_F32 ? 8 : 4;
    const unsigned padx = self ? (unsigned)(16 / es) : 0u;
    if (!encode || ((size_t)L.nx * es) % 16 != 0) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny, (cuuint64_t)L.nz, (cuuint64_t)Q};
    const cuuint64_t strides[3] = {(cuuint64_t)L.nx * es, (cuuint64_t)L.nx * L.ny * es, (cuuint64_t)L.S * es};
    const cuuint32_t box[4] = {(cuuint32_t)(TX + 2 * padx), (cuuint32_t)(self ? ty + 2 : ty), 1, Q};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = es == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
    return encode(map, dt, 4, f, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

FusedOfs fused_offsets(const Lat &L)
{
    FusedOfs ofs;
    for (int i = 0; i < Q; i++) {
        const long long o = (long long)i * L.S;
        const long long d = cx(i) + (long long)cy(i) * L.nx + (long long)cz(i) * L.nx * L.ny;
        ofs.pop[i] = o;
        ofs.push[i] = o + d;
        // slot 0 never pushes; the others lie at least S - nx*ny - nx - 1 > 0
        // above the array base
        ofs.pop32[i] = (unsigned)o;
        ofs.push32[i] = (unsigned)(o + d);
    }
    return ofs;
}

// The 32-bit offsets hold every store: the highest is slot 18 of the pushed
// neighbour plus a periodic wrap of N.
bool fused_rel32(const Lat &L)
{
    return !L.wide && (long long)Q * L.S + 2LL * L.N + (long long)L.nx * L.ny + L.nx + 1 < (1LL << 32);
}

template <class S, int TY, bool GEN, bool SELF, bool TMA, bool R32>
static void launch_cfg(const Lat &L, const void *fin, void *fout, const float *psi, const uint8_t *type,
                       const CUtensorMap &tm, int zc, int wait_limit, cudaStream_t s)
{
    using C = Cfg<S, TY, GEN, SELF>;
    using P = typename S::P;
    auto kern = k_fused<S, TY, GEN, SELF, TMA, R32>;
    static bool configured = false;  // the attribute is per function and process
    if (!configured) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::bytes);
        configured = true;
    }
    dim3 grid((L.nx + TX - 1) / TX, (L.ny + TY - 1) / TY, (L.nz + zc - 1) / zc);
    kern<<<grid, C::NT, C::bytes, s>>>(L, (const P *)fin, (P *)fout, psi, type, zc, fused_offsets(L), tm, wait_limit);
}

// Configurations built, each with ψ formed in the kernel (SELF) or from
// memory: τ = 1 with 32-bit offsets at 4 or 8 rows per tile (TMA) or 8
// (loads); any τ with 32- or 64-bit offsets at 8 rows (also taken by τ = 1
// lattices that need 64-bit offsets: same results).
template <class S, bool SELF>
static void launch_fused_t(const Lat &L, const void *fin, void *fout, const float *psi, const uint8_t *type,
                           const CUtensorMap *tmap, cudaStream_t s, int zc, int ty, int wait_limit)
{
    const CUtensorMap none{};
    const CUtensorMap &tm = tmap ? *tmap : none;
    const bool r32 = fused_rel32(L), tau1 = fused_tau1(L) && r32;
    if (tau1) {
        if (tmap && ty == 4)
            launch_cfg<S, 4, false, SELF, true, true>(L, fin, fout, psi, type, tm, zc, wait_limit, s);
        else if (tmap)
            launch_cfg<S, 8, false, SELF, true, true>(L, fin, fout, psi, type, tm, zc, wait_limit, s);
        else
            launch_cfg<S, 8, false, SELF, false, true>(L, fin, fout, psi, type, tm, zc, wait_limit, s);
    } else if (r32) {
        if (tmap)
            launch_cfg<S, 8, true, SELF, true, true>(L, fin, fout, psi, type, tm, zc, wait_limit, s);
        else
            launch_cfg<S, 8, true, SELF, false, true>(L, fin, fout, psi, type, tm, zc, wait_limit, s);
    } else {
        if (tmap)
            launch_cfg<S, 8, true, SELF, true, false>(L, fin, fout, psi, type, tm, zc, wait_limit, s);
        else
            launch_cfg<S, 8, true, SELF, false, false>(L, fin, fout, psi, type, tm, zc, wait_limit, s);
    }
}

int fused_rows(const Lat &L, int ty_request, bool tma)
{
    // only the τ = 1 configurations with TMA come in two heights
    return (ty_request == 4 && tma && fused_tau1(L) && fused_rel32(L)) ? 4 : 8;
}

void launch_fused(int storage, const Lat &L, const void *fin, void *fout, const float *psi, const uint8_t *type,
                  const CUtensorMap *tmap, cudaStream_t s, int zc, int ty, int wait_limit, bool self)
{
    const int rows = fused_rows(L, ty, tmap != nullptr);
    if (zc <= 0) zc = fused_zchunk(L, rows);
    if (zc > L.nz) zc = L.nz;
    if (self)
        LBE_DISPATCH(storage, (launch_fused_t<S, true>(L, fin, fout, psi, type, tmap, s, zc, rows, wait_limit)));
    else
        LBE_DISPATCH(storage, (launch_fused_t<S, false>(L, fin, fout, psi, type, tmap, s, zc, rows, wait_limit)));
}

template <class S>
static void launch_fused_batch_t(const BatchIndex &B, int total, int ctas, cudaStream_t s)
{
    using C = Cfg<S, BATCH_TY, true, false>;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_fused_batch<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::bytes);
        configured = true;
    }
    k_fused_batch<S><<<ctas, C::NT, C::bytes, s>>>(B, total);
}

void launch_fused_batch(int storage, const BatchIndex &B, int total_tiles, int ctas, cudaStream_t s)
{
    LBE_DISPATCH(storage, (launch_fused_batch_t<S>(B, total_tiles, ctas, s)));
}

int fused_batch_ctas_per_sm(int storage)
{
    int n = 0;
    LBE_DISPATCH(storage, (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused_batch<S>, TX * BATCH_TY,
                                                                         Cfg<S, BATCH_TY, true, false>::bytes)));
    return n > 0 ? n : 1;
}

}  // namespace lbe
