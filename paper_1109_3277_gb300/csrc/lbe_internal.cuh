// Internal declarations shared by the CUDA translation units of liblbe.
// Method: §2 of Günther et al., arXiv:1109.3277 (two-component Shan–Chen
// D3Q19 BGK lattice Boltzmann with rigid ellipsoids).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/lbe.h"

namespace lbe {

constexpr int Q = 19;
constexpr uint8_t FLUID = 0, WALL = 1, PART = 2;
constexpr uint32_t NONE = 0xFFFFFFFFu;

// D3Q19 velocity set (§2): rest, the 6 axis directions, the 12 face
// diagonals; the opposite of direction i is i+1 for odd i and i-1 for even i.
__host__ __device__ constexpr int cx(int i)
{
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int cy(int i)
{
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int cz(int i)
{
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float wgt(int i) { return i == 0 ? 1.f / 3.f : (i < 7 ? 1.f / 18.f : 1.f / 36.f); }
__host__ __device__ constexpr double wgtd(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

// Population storage.  FP32 stores f itself; the 16-bit modes store
// δf = f - w_i ρ_ref^c (the offset from the rest equilibrium at ρ_ref).
// The two components of one direction at one node sit side by side: the
// population array is P[19][S] with P = (red, blue) of the storage type, so
// element (c, i, n) lies at 2 (i S + n) + c in units of T.  One 32-bit
// (16-bit modes) or 64-bit (FP32) access moves both components.
// raw2/enc2 convert a pair of stored quantities (δf, or f for FP32) to and
// from FP32; ld2f/st2f add and subtract the slot's base (w_i ρ_ref^c, 0 in
// FP32); raw/enc convert one scalar element.
struct StF32 {
    using T = float;
    using P = float2;
    static __device__ __forceinline__ float raw(T v) { return v; }
    static __device__ __forceinline__ T enc(float v) { return v; }
    static __device__ __forceinline__ float2 raw2(P v) { return v; }
    static __device__ __forceinline__ P enc2(float2 v) { return v; }
};
struct StF16 {
    using T = __half;
    using P = __half2;
    static __device__ __forceinline__ float raw(T v) { return __half2float(v); }
    static __device__ __forceinline__ T enc(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ float2 raw2(P v) { return __half22float2(v); }
    static __device__ __forceinline__ P enc2(float2 v) { return __floats2half2_rn(v.x, v.y); }
};
// BF16 keeps 8 significant bits.  Rounding a population's offset to nearest
// would bias the flow: in a demixed fluid the offsets are ~0.6 w_i, whose
// half-ulp (~1e-4) is of the order of the velocity part 3 w_i ρ c·u, and
// the same values round the same way step after step.  The pairs are
// therefore rounded up with probability equal to the discarded fraction
// (unbiased): a 16-bit increment, taken from a hash of the pair's own FP32
// bits, is added to each value's bit pattern before truncation.  The hash
// makes the result a fixed function of the value (runs and batches stay
// bit-identical), and over the values a node sees it acts as a uniform
// random increment.
__device__ __forceinline__ uint32_t mix32(uint32_t a, uint32_t b)
{
    uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return h;
}
__device__ __forceinline__ uint16_t bf16_unbiased(float v, uint32_t r16)
{
    const uint32_t b = __float_as_uint(v);
    if ((b & 0x7F800000u) == 0x7F800000u) return (uint16_t)(b >> 16);  // inf, NaN: truncated
    return (uint16_t)((b + r16) >> 16);  // carries into the exponent are the correct round-up
}
struct StBF16 {
    using T = __nv_bfloat16;
    using P = __nv_bfloat162;
    static __device__ __forceinline__ float raw(T v) { return __bfloat162float(v); }
    static __device__ __forceinline__ T enc(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float2 raw2(P v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ P enc2(float2 v)
    {
        const uint32_t h = mix32(__float_as_uint(v.x), __float_as_uint(v.y));
        __nv_bfloat162_raw r;
        r.x = bf16_unbiased(v.x, h & 0xFFFFu);
        r.y = bf16_unbiased(v.y, h >> 16);
        return P(r);
    }
};

// Lattice parameters passed by value to every kernel.
struct Lat {
    int nx, ny, nz, walls;
    int N;                 // nodes (< 2^31)
    long long S;           // pairs per direction array (>= N, padded so the 19
                           // arrays are not a power of two apart)
    float tau[2], itau[2];
    float g;
    float body[3];
    float base[2][Q];      // w_i ρ_ref^c for the 16-bit modes, 0 for FP32
    float rref[2];         // ρ_ref^c for the 16-bit modes, 0 for FP32
    double rho_ref[2];
    int np;                        // particles (bounds checks)
    int wide;                      // 1: the fused kernel takes 64-bit store offsets
    unsigned *status;              // bit 0: a TMA copy of the fused kernel never completed
    unsigned long long *err;       // bounds-check record (checked builds only)
};

// Pair index of direction i at node n (units of the storage's pair type).
__host__ __device__ __forceinline__ size_t pidx(const Lat &L, int i, long long n)
{
    return (size_t)i * (size_t)L.S + (size_t)n;
}

// Base (w_i ρ_ref^red, w_i ρ_ref^blue) of direction i: f = stored + base.
__device__ __forceinline__ float2 base2(const Lat &L, int i) { return make_float2(L.base[0][i], L.base[1][i]); }

// f of both components of slot i at node n, and the store of f.
template <class S>
__device__ __forceinline__ float2 ld2f(const typename S::P *f, const Lat &L, int i, long long n)
{
    const float2 v = S::raw2(f[pidx(L, i, n)]);
    return make_float2(L.base[0][i] + v.x, L.base[1][i] + v.y);
}
template <class S>
__device__ __forceinline__ void st2f(typename S::P *f, const Lat &L, int i, long long n, float2 v)
{
    f[pidx(L, i, n)] = S::enc2(make_float2(v.x - L.base[0][i], v.y - L.base[1][i]));
}

// Densities ρ are kept per node as (red, blue) pairs: the array rho is
// float2 [N] (passed as float *), so one 8-byte access moves both
// components.  ψ stays psi[2][N] (one array per component): the fused
// kernel's ring copies each component's ψ into its place in the (ψ_b, ψ_r)
// ring pair, which measured faster at 512^3 than copying an interleaved
// pair.
__host__ __device__ __forceinline__ float2 ld_pair(const float *a, long long n)
{
    return reinterpret_cast<const float2 *>(a)[n];
}
__host__ __device__ __forceinline__ void st_pair(float *a, long long n, float2 v)
{
    reinterpret_cast<float2 *>(a)[n] = v;
}

// The order in which a node's 19 stored quantities are summed: the nine
// opposite pairs p_k = d_{2k+1} + d_{2k+2} first, then a balanced tree
// ((p0 + p1) + (p2 + p3)) + ((p4 + p5) + (p6 + p7)) + (p8 + d0), each
// addition rounded to nearest per component.  Every kernel that sums a
// node's populations (the density kernel, the shell fill, the fused
// kernel's moments) takes this order, so they agree bit for bit; the tree
// keeps the chain of dependent additions five deep.  The pair sums are fed
// in k order as they are formed (put), so that few stay live.
struct FaddLanes {
    __device__ __forceinline__ float2 operator()(float2 a, float2 b) const
    {
        return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
    }
};
struct PairTree {
    float2 h, a, b;
    template <class ADD>
    __device__ __forceinline__ void put(int k, float2 p, ADD add)
    {
        if (k == 0 || k == 2 || k == 4 || k == 6 || k == 8) {
            h = p;
            return;
        }
        const float2 q = add(h, p);
        if (k == 1) a = q;
        if (k == 3) a = add(a, q);
        if (k == 5) b = q;
        if (k == 7) b = add(b, q);
    }
    template <class ADD>
    __device__ __forceinline__ float2 finish(float2 d0, ADD add) const
    {
        return add(add(a, b), add(h, d0));
    }
};

// Densities (ρ^red, ρ^blue) of node n from its stored populations: the
// stored quantities summed in the order above, then ρ_ref added (0 in
// FP32).  Every kernel that needs a node's density from memory takes it
// from here.
template <class S>
__device__ __forceinline__ float2 node_rho2(const typename S::P *__restrict__ f, const Lat &L, long long n)
{
    PairTree t;
#pragma unroll
    for (int k = 0; k < 9; k++)
        t.put(k, FaddLanes{}(S::raw2(f[pidx(L, 2 * k + 1, n)]), S::raw2(f[pidx(L, 2 * k + 2, n)])), FaddLanes{});
    const float2 a = t.finish(S::raw2(f[pidx(L, 0, n)]), FaddLanes{});
    return make_float2(__fadd_rn(L.rref[0], a.x), __fadd_rn(L.rref[1], a.y));
}

// Checked builds (-DLBE_CHECK) verify every data-dependent or computed index
// before use; a bad one is recorded (code << 40 | index) and the access is
// skipped.  Release builds compile the checks away.
#ifdef LBE_CHECK
__device__ __forceinline__ bool idx_ok(const Lat &L, long long i, long long lim, int code)
{
    if (i >= 0 && i < lim) return true;
    atomicCAS(L.err, 0ull, ((unsigned long long)code << 40) | ((unsigned long long)i & 0xFFFFFFFFFFull));
    return false;
}
#else
__device__ __forceinline__ bool idx_ok(const Lat &, long long, long long, int) { return true; }
#endif

// Particle state on the device (structure of arrays, FP64).
struct Parts {
    int n;
    double *X, *q, *V, *W;          // position [3n], quaternion [4n], velocity, ω (lab)
    double *Xold, *qold;            // geometry before the last update
    double *rp, *ro, *drho;         // radii, colour Δρ
    double *M, *Ipar, *Iperp;       // mass and body-frame inertia
    double *Flink, *Tlink;          // momentum exchange of the current step
    double *Fpair, *Tpair;          // pair forces of the current step
    double *Fpend, *Tpend;          // fill/empty momentum for the next update
    double *F, *T;                  // total of the last update
    unsigned long long *fix;        // [6n] link force and torque in 2^-40 fixed point
    int nsplit;                     // pair-force splits of the j range
    double *ppart;                  // [nsplit][6][n] pair-force partial sums
    float4 *X32;                    // FP32 (x, y, z, max radius) for the pair prefilter
    float4 *K32;                    // FP32 velocity [2p] and ω [2p+1] for the fused links
    void *geo;                      // per particle: coverage geometry of the last and the current update
};

// Particle nodes next to fluid nodes, collected each step by the shell-fill
// kernel: entry (particle node s, mask of the directions j whose neighbour
// s + c_j is a fluid node).  A node enters at most once per step, so cap = N
// cannot overflow.
struct LinkList {
    uint2 *ent;   // [cap]
    int *count;   // entries this step (reset before the density kernel)
    int cap;
};

constexpr double FIXED_UNIT = 1.0 / 1099511627776.0;  // 2^-40

// Shell fill of solid node n (Eq. 10 and the colour rule): the mean ρ^c of
// its fluid neighbours, the colour Δρ added to red if positive, else |Δρ| to
// blue, then ψ^c = 1 - exp(-ρ^c).  Nothing for a node without a fluid
// neighbour (never read by a fluid node).  nb(i) is the neighbour index
// along c_i, -1 beyond a wall; rho_of(m) gives (ρ^red, ρ^blue) of fluid node
// m.  Returns the mask of fluid neighbours.
template <class NB, class RHO>
__device__ __forceinline__ uint32_t shell_fill_with(const Lat &L, float *__restrict__ psi,
                                                    const uint8_t *__restrict__ type, int n, float dr, NB nb,
                                                    RHO rho_of)
{
    float s0 = 0.f, s1 = 0.f;
    int cnt = 0;
    uint32_t fm = 0;
#pragma unroll
    for (int i = 1; i < Q; i++) {
        const int m = nb(i);
        if (m < 0 || type[m] != FLUID) continue;
        const float2 r = rho_of(m);
        s0 += r.x;
        s1 += r.y;
        cnt++;
        fm |= 1u << i;
    }
    if (cnt == 0) return 0;
    float r0 = s0 / (float)cnt, r1 = s1 / (float)cnt;
    if (dr > 0.f)
        r0 += dr;
    else
        r1 += fabsf(dr);
    psi[n] = 1.f - expf(-r0);
    psi[(size_t)L.N + n] = 1.f - expf(-r1);
    return fm;
}

// The same with the neighbours' densities from the array rho[2][N].
template <class NB>
__device__ __forceinline__ uint32_t shell_fill(const Lat &L, const float *__restrict__ rho, float *__restrict__ psi,
                                               const uint8_t *__restrict__ type, int n, float dr, NB nb)
{
    return shell_fill_with(L, psi, type, n, dr, nb,
                           [&](int m) { return ld_pair(rho, m); });
}

// Append (n, m) for the lanes with m != 0 to a link list: one atomic per
// warp.  Called by all 32 lanes.
__device__ __forceinline__ void append_links(const LinkList &ll, int n, uint32_t m)
{
    const unsigned want = __ballot_sync(0xffffffffu, m != 0);
    if (!want) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(want) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(ll.count, __popc(want));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (m) {
        const int k = base + __popc(want & ((1u << lane) - 1u));
        if (k < ll.cap) ll.ent[k] = make_uint2((unsigned)n, m);
    }
}

// Cell list of the particles for the pair forces: cubic-ish cells of edge
// >= the largest pair reach, so a particle's partners lie in its own cell
// and the 26 around it.
struct Cells {
    int n[3];          // cells per axis
    float inv[3];      // cells per lattice unit
    int ncell;
    int *count;        // [ncell] particles per cell
    int *start;        // [ncell + 1] exclusive prefix
    int *fill;         // [ncell] fill cursor
    int *idx;          // [cap] particle indices by cell
    int *cid;          // [cap] cell of each particle
};

// Pair offsets of the fused kernel's loads and stores from a node: its own
// slot pop[i] = i S and the neighbour's it pushes to, push[i] = pop[i] +
// (cx + cy nx + cz nx ny), so the address of a load or of an interior push
// is one add; as 64-bit words, and as 32-bit words (pop32, push32) used
// where they fit (fused_rel32).
struct FusedOfs {
    long long pop[Q];
    long long push[Q];
    unsigned pop32[Q];
    unsigned push32[Q];
};
FusedOfs fused_offsets(const Lat &L);
bool fused_rel32(const Lat &L);

struct Pair {
    double k_hertz, lub_cut, mu;
    int mode;
};

// One lattice of a batch (all boxes step together in multi-lattice kernels).
// Ping-pong parities live in a device array beside the table, so that a
// captured step can be replayed whatever the parity.
struct BoxDev {
    CUtensorMap tmap[2];     // population planes of f[0], f[1] (when tma)
    int tma;                 // the fused kernel stages planes by TMA
    Lat L;
    FusedOfs ofs;
    void *f[2];
    float *rho, *psi;
    uint8_t *type;
    uint32_t *owner[2];
    Parts P;                 // nsplit = 1 inside a batch
    Pair pair;
    int mode;                // particle mode
    LinkList links;          // link nodes of this box (ent null without particles)
    int zc, ntx, nty, nzc;   // fused-kernel tiling of this box
};

// Prefix offsets of the boxes' work items (tiles, nodes, particles).
struct BatchIndex {
    const BoxDev *box;
    int nbox;
    const int *tile0, *node0, *part0;   // [nbox + 1]
    int *par;                           // [2 nbox]: cur, ocur
    int *counter;                       // persistent tile queue of the fused kernel
};

// ---- launchers (fluid.cu) -------------------------------------------------
void launch_init_f(int storage, const Lat &L, const double *rho0, void *f, const uint8_t *type,
                   cudaStream_t s);
void launch_moments(int storage, const Lat &L, const void *f, const uint8_t *type, float *rho,
                    float *psi, cudaStream_t s);
void launch_rho(int storage, const Lat &L, const void *f, const uint8_t *type, float *rho, float *psi,
                cudaStream_t s);
void launch_shell(const Lat &L, const float *rho, float *psi, const uint8_t *type,
                  const uint32_t *owner, const double *drho, const LinkList &ll, cudaStream_t s);
// Shell fill of the particles' own nodes (one CTA per particle over its
// candidate rows) and of the wall planes: the solid nodes a fluid node can
// see, without a sweep of the lattice.
// Shell fill of the particles' own nodes (one CTA per particle over its
// candidate rows), with the neighbours' densities from rho, and of the wall
// planes, with the densities of the planes next to the walls computed from
// the populations f (a lattice without particles runs no density kernel).
void launch_shell_particles(const Lat &L, const Parts &P, const float *rho, float *psi, const uint8_t *type,
                            const uint32_t *owner, const LinkList &ll, cudaStream_t s);
void launch_shell_walls(int storage, const Lat &L, const void *f, float *psi, const uint8_t *type, cudaStream_t s);
void launch_collide_stream(int storage, const Lat &L, const void *fin, void *fout, const float *psi,
                           const uint8_t *type, cudaStream_t s);
void launch_fields(int storage, const Lat &L, const void *f, const float *psi, const uint8_t *type,
                   double *rho_out, double *vel_out, cudaStream_t s);
void launch_mass(int storage, const Lat &L, const void *f, const uint8_t *type, double *partials,
                 int nblocks, double *out, cudaStream_t s);
void launch_get_f(int storage, const Lat &L, const void *f, double *out, cudaStream_t s);
void launch_set_f(int storage, const Lat &L, const double *in, void *f, cudaStream_t s);
int mass_blocks();

// ---- batched launchers (one launch steps every box of a batch) -------------
void launch_rho_batch(int storage, const BatchIndex &B, int total_nodes, cudaStream_t s);
void launch_shell_batch(const BatchIndex &B, int total_nodes, cudaStream_t s);
void launch_fused_batch(int storage, const BatchIndex &B, int total_tiles, int ctas, cudaStream_t s);
int fused_batch_ctas_per_sm(int storage);
void launch_pairs_batch(const BatchIndex &B, int total_parts, cudaStream_t s);
void launch_integrate_batch(const BatchIndex &B, int total_parts, cudaStream_t s);
void launch_geom_batch(const BatchIndex &B, int total_parts, cudaStream_t s);
void launch_claim_batch(const BatchIndex &B, int total_parts, cudaStream_t s);
void launch_transition_batch(int storage, const BatchIndex &B, int total_parts, cudaStream_t s);
void launch_reset_batch(const BatchIndex &B, int total_parts, cudaStream_t s);
void launch_batch_quat(const BatchIndex &B, double *out, cudaStream_t s);
void launch_link_batch(int storage, const BatchIndex &B, cudaStream_t s);
void launch_flip_batch(const BatchIndex &B, cudaStream_t s);

// ---- launchers (fused.cu) -------------------------------------------------
// The fused kernel's tiles are 32 nodes wide and 4 or 8 rows high; zc is the
// z chunk in planes (0: the default for the lattice), ty the requested tile
// height (4 or 8; configurations without a 4-row variant take 8), and
// wait_limit the tries of each bounded wait for a box copy.
constexpr int FUSED_TX = 32, FUSED_TY_BATCH = 8;
constexpr int FUSED_WAIT_LIMIT = 1 << 22;
// self: the kernel forms ψ of fluid nodes from the densities of the tile
// and a one-node halo (psi then holds ψ of solid nodes only); otherwise psi
// holds ψ of every node (density kernel and shell fill).
void launch_fused(int storage, const Lat &L, const void *fin, void *fout, const float *psi, const uint8_t *type,
                  const CUtensorMap *tmap, cudaStream_t s, int zc, int ty, int wait_limit, bool self);
int fused_zchunk(const Lat &L, int ty);
// The tile height launch_fused takes for a request (4 only where built).
int fused_rows(const Lat &L, int ty_request, bool tma);
bool fused_tau1(const Lat &L);
// Tensor map of one population buffer for the fused kernel's box copies
// (tile plus a one-node halo, x widened to 16-byte boundaries: 40 x (ty+2) x
// 1 x 19 pairs at 16 bit, 36 x (ty+2) x 1 x 19 in FP32, of the (x, y, z,
// direction) array); false if the lattice's row pitch is not a multiple of
// 16 bytes or the driver lacks the call.
// self: the box with the halo; otherwise the tile alone (32 x ty x 1 x 19).
bool fused_plane_map(CUtensorMap *map, void *f, const Lat &L, int storage, int ty, bool self);

// Box lookup: the box b with off[b] <= i < off[b+1] (binary search).
__device__ __forceinline__ int find_box(const int *off, int nbox, int i)
{
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---- launchers (particles.cu) ---------------------------------------------
void launch_links(int storage, const Lat &L, const Parts &P, void *fnew, const float *rho,
                  const uint8_t *type, const uint32_t *owner, cudaStream_t s);
void launch_link(int storage, const Lat &L, const LinkList &ll, const float *rho, const uint32_t *owner,
                 const Parts &P, void *fout, cudaStream_t s);
void launch_pairs(const Lat &L, const Parts &P, const Pair &pp, const Cells &C, cudaStream_t s);
void launch_integrate(const Lat &L, const Parts &P, int mode, cudaStream_t s);
// Coverage geometry of the particles (old and current), once per update;
// geom_bytes_per_particle() is the size of one particle's record.
void launch_geom(const Lat &L, const Parts &P, cudaStream_t s);
size_t geom_bytes_per_particle();
void launch_claim(const Lat &L, const Parts &P, int first, uint32_t *owner_new, cudaStream_t s);
void launch_transition(int storage, const Lat &L, const Parts &P, void *f, uint8_t *type,
                       const uint32_t *owner_old, const uint32_t *owner_new, int placement,
                       cudaStream_t s);
void launch_reset(const Lat &L, const Parts &P, int use_old, uint32_t *owner, cudaStream_t s);
void launch_verify(const Lat &L, const uint8_t *type, const uint32_t *owner, cudaStream_t s);

}  // namespace lbe
