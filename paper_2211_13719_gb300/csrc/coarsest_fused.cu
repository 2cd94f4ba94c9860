// The coarsest level's GMRES cycle in one persistent kernel: the coarsest
// solve of the V-cycle (Sec. 8), GMRES(m) from x = 0 on the 9-point coarse
// operator (Sec. 6), with the operator applied on the tensor cores as in
// coarse_tc.cu.
//
// On the coarsest lattice (a few hundred sites; fields of a few MB that stay
// in L2) each GMRES step of the launch-per-operation path is about seven
// dependent launches -- input scale and packing, the tensor-core stencil,
// the Arnoldi dots, the subtract-and-normalise, a norm fix-up, the Givens
// update -- each bound by its launch and its grid-wide reduction, not by the
// bytes it moves.  Here one cooperative launch runs the whole cycle:
//
//  * One 512-thread CTA per SM, all resident at once (a kernel that holds
//    tensor memory is resident one CTA per SM for the occupancy calculator
//    and the cooperative launch), each owning one or two coarse sites.  A
//    CTA owns its sites' 64 rows of every field, so the Krylov basis never
//    crosses CTAs.  What does: the packed 16-bit image of the newest basis
//    vector (the stencil's neighbour input), per-CTA partial sums, and
//    per-RHS scalars.
//  * The stencil of a step is the tcgen05 MMA of the coarse stencil kernel:
//    link and neighbour tiles through a bulk-copy ring, FP32 accumulation in
//    tensor memory (one accumulator per own site) allocated once for the
//    launch.  Each own site has its own copy ring and issuing thread.  The
//    result, scaled to w = A v_j, stays in shared memory for the dots and the
//    update of the same step.  While the stencils stream, another warp does
//    the Givens update of the previous column.
//  * Grid-wide barriers (a monotonic arrival counter; every wait bounded)
//    separate the three phases of a step: (1) stencil + partial dots,
//    (2) the sum of the partials of each RHS column by the column's owner
//    CTA, (3) subtract, pack the next image, partial norms.
//  * The Givens rotations, the back substitution and the per-RHS scalars
//    run in FP64 in the owner CTA of each column.
//
// Two numerical choices differ from the launch-per-operation path:
//  * The norm of each new basis vector is summed from its components (one
//    more set of partials per step) instead of taken from the Pythagorean
//    identity, so no fix-up pass exists.
//  * The 16-bit image of a new, not yet normalised basis vector u is scaled
//    by 256 / ||w||, with w the stencil output u was orthogonalised from.
//    Since |u_i| <= ||u|| <= ||w||, every image component is at most 256
//    in magnitude; the separate maximum-finding pass is not needed.
//
// Every wait is bounded: the mbarrier waits of the bulk-copy ring and the
// MMAs as in the stencil kernel, and the grid barriers.  A CTA whose wait
// expires records an error (the level's tensor-core error flag, read by the
// solve, and an abort word the other CTAs poll), drains its own copies and
// MMAs, frees its tensor memory and returns; the others stop at their next
// barrier.
#include "mg.cuh"
#include "tc_common.cuh"

namespace mrhs {

namespace {

using namespace tc;

constexpr int NC = 64;                  // coarse dof
constexpr int MROWS = 128;              // 2 * NC real rows of a link tile
constexpr int A_TILE = MROWS * NC * 2;  // bytes of one 16-bit link tile
constexpr int RING = 3;                 // bulk-copy ring depth of each own site (one ring and thread per site)
constexpr int MMAX = 16;                // largest restart length
constexpr int THREADS = 512;            // 16 warps: the row phases are bound by L2 latency
constexpr int MAX_SITES = 2;            // most coarse sites of one CTA (each staged in shared memory)
constexpr uint32_t BAR_LIMIT = 1u << 22;  // polls of a grid barrier before it gives up
constexpr float IMG_BOUND = 256.f;        // largest image component

struct FusedArgs {
    int L[4];
    int G;                   // CTAs; CTA c owns the sites c, c + G, c + 2G, ... below V
    int V;                   // coarse sites
    int S;                   // most sites of one CTA
    int cols_site;           // tensor-memory columns of one site's accumulator
    int n, npad, m;
    uint32_t idesc, tmem_cols, b_tile, stage_bytes;
    const uint8_t *Abf;      // link tiles [V][9], A_TILE bytes each
    const float *lscale;     // per-site link scale [V]
    uint8_t *img;            // packed image of the newest basis vector [V] x b_tile
    const float2 *b;         // right-hand side [V][64][n]
    float2 *x;               // solution [V][64][n]
    float2 *Vb;              // basis, m + 1 fields [V][64][n]
    double2 *part;           // [G][m + 1][n]: <v_i, w> (i <= j), then (||w||^2, 0) at i = j + 1
    double *npart;           // [G][n]: ||u||^2 of the newest basis vector, per CTA
    double2 *hcol;           // [m + 1][n]: the current Arnoldi column
    float *sig;              // [n]: scale of the current image
    double2 *R;              // [n][m + 1][m] rotated Hessenberg
    double *cs;              // [n][m]
    double2 *sn;             // [n][m]
    double2 *g;              // [n][m + 1]
    double2 *y;              // [m][n]
    unsigned *sync;          // [0]: barrier arrivals, [1]: abort word; zero at launch
    int *err;                // the level's tensor-core error flag
    uint32_t first_limit;    // try_wait rounds of the first operand wait (0: a test expires it)
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// order this thread's generic-proxy global writes before later async-proxy (bulk copy) reads
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

__device__ __forceinline__ void record_error(const FusedArgs &a) {
    atomicExch(a.err, 1);
    atomicExch(a.sync + 1, 1u);
}

// Grid-wide barrier number k: every CTA adds one arrival and waits until the
// counter reaches (k + 1) * G.  Gives up after BAR_LIMIT polls, or as soon as
// another CTA has recorded an error.  False: the CTA must stop.
__device__ bool grid_barrier(const FusedArgs &a, unsigned &k, int *flag_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(a.sync, 1u);
        const unsigned target = (k + 1) * (unsigned)a.G;
        bool ok = true;
        uint32_t it = 0;
        while (ld_acquire_u32(a.sync) < target) {
            if (ld_relaxed_u32(a.sync + 1) != 0u || ++it > BAR_LIMIT) {
                ok = false;
                break;
            }
            __nanosleep(20);
        }
        if (!ok) record_error(a);
        __threadfence();
        *flag_sh = ok ? 0 : 1;
    }
    ++k;
    __syncthreads();
    return *flag_sh == 0;
}

// thread -> (RHS column, row slice): RS = THREADS / n slices of the site's 64 rows
struct RowMap {
    int r, sub, RS;
    bool active;
    __device__ RowMap(int n) {
        RS = THREADS / n;
        r = threadIdx.x % n;
        sub = threadIdx.x / n;
        active = sub < RS;
    }
};

// eta[r] = sqrt(sum over CTAs of npart[c][r]), summed in CTA order (identical in every CTA)
__device__ void reduce_norms(const FusedArgs &a, double *red_d, double *eta) {
    const RowMap t(a.n);
    if (t.active) {
        double s = 0.0;
        #pragma unroll 8
        for (int c = t.sub; c < a.G; c += t.RS) s += a.npart[(int64_t)c * a.n + t.r];
        red_d[t.sub * a.n + t.r] = s;
    }
    __syncthreads();
    if ((int)threadIdx.x < a.n) {
        double s = 0.0;
        for (int q = 0; q < t.RS; ++q) s += red_d[q * a.n + threadIdx.x];
        eta[threadIdx.x] = sqrt(fmax(s, 0.0));
    }
    __syncthreads();
}

// Givens update of column jc of RHS r (one thread): col = hcol[0..jc][r], h_{jc+1,jc} = beta
__device__ void givens_column(const FusedArgs &a, int r, int jc, double beta) {
    const int m = a.m;
    double2 col[MMAX + 1];
    for (int i = 0; i <= jc; ++i) col[i] = a.hcol[(int64_t)i * a.n + r];
    col[jc + 1] = make_double2(beta, 0.0);
    for (int i = 0; i < jc; ++i) {
        const double c = a.cs[(int64_t)r * m + i];
        const double2 s = a.sn[(int64_t)r * m + i];
        const double2 p = col[i], q = col[i + 1];
        col[i] = make_double2(c * p.x + s.x * q.x - s.y * q.y, c * p.y + s.x * q.y + s.y * q.x);
        col[i + 1] = make_double2(-(s.x * p.x + s.y * p.y) + c * q.x, -(s.x * p.y - s.y * p.x) + c * q.y);
    }
    const double2 p = col[jc], q = col[jc + 1];
    const double np = hypot(p.x, p.y), nq = hypot(q.x, q.y);
    double c;
    double2 s;
    if (nq == 0.0) {
        c = 1.0;
        s = make_double2(0.0, 0.0);
    } else if (np == 0.0) {
        c = 0.0;
        s = make_double2(q.x / nq, -q.y / nq);
    } else {
        const double t = hypot(np, nq);
        c = np / t;
        const double2 ph = make_double2(p.x / np, p.y / np);
        const double2 cq = make_double2(q.x / t, -q.y / t);
        s = make_double2(ph.x * cq.x - ph.y * cq.y, ph.x * cq.y + ph.y * cq.x);
    }
    a.cs[(int64_t)r * m + jc] = c;
    a.sn[(int64_t)r * m + jc] = s;
    col[jc] = make_double2(c * p.x + s.x * q.x - s.y * q.y, c * p.y + s.x * q.y + s.y * q.x);
    for (int i = 0; i <= jc; ++i) a.R[((int64_t)r * (m + 1) + i) * m + jc] = col[i];
    double2 *g = a.g + (int64_t)r * (m + 1);
    const double2 gj = g[jc];
    g[jc] = make_double2(c * gj.x, c * gj.y);
    g[jc + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
}

// y = R^-1 g for RHS r (one thread), the leading m x m triangle
__device__ void back_substitute(const FusedArgs &a, int r) {
    const int m = a.m;
    double2 yy[MMAX];
    for (int i = m - 1; i >= 0; --i) {
        double2 acc = a.g[(int64_t)r * (m + 1) + i];
        for (int l = i + 1; l < m; ++l) {
            const double2 rv = a.R[((int64_t)r * (m + 1) + i) * m + l];
            acc.x -= rv.x * yy[l].x - rv.y * yy[l].y;
            acc.y -= rv.x * yy[l].y + rv.y * yy[l].x;
        }
        const double2 d = a.R[((int64_t)r * (m + 1) + i) * m + i];
        const double dd = d.x * d.x + d.y * d.y;
        yy[i] = dd > 0.0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                         : make_double2(0.0, 0.0);
    }
    for (int i = 0; i < m; ++i) a.y[(int64_t)i * a.n + r] = yy[i];
}

// One issuing thread per own site: the 9 direction tiles of that site's
// stencil through the site's own ring (its stages at `sbase`, its barriers at
// full0 / empty0) and the MMAs into its tensor-memory accumulator `acc`, then
// a commit on `done` (which expects one commit per own site).  q0: the ring
// position of the site's first load, continued across steps.  On an expired
// wait the loads in flight are drained (every one is in its own stage, so its
// parity is exact).
__device__ bool stencil_issue(const FusedArgs &a, int64_t site, uint32_t sbase, uint32_t full0, uint32_t empty0,
                              uint32_t done, uint32_t acc, uint32_t &q0) {
    bool ok = true;
    int issued = 0, consumed = 0;
    for (int step = 0; step < 9 + RING - 1 && ok; ++step) {
        if (step < 9) {
            const uint32_t q = q0 + step, s = q % RING;
            if (q >= (uint32_t)RING) ok = mbar_wait(empty0 + 8 * s, ((q / RING) - 1) & 1);
            if (!ok) break;
            const int64_t nb = stencil_nb_site(site, a.L, step);
            const uint32_t sa = sbase + s * a.stage_bytes;
            mbar_expect_tx(full0 + 8 * s, A_TILE + a.b_tile);
            bulk_g2s(sa, a.Abf + ((size_t)site * 9 + step) * A_TILE, A_TILE, full0 + 8 * s);
            bulk_g2s(sa + A_TILE, a.img + (size_t)nb * a.b_tile, a.b_tile, full0 + 8 * s);
            ++issued;
        }
        const int e = step - (RING - 1);
        if (e >= 0 && e < 9) {
            const uint32_t q = q0 + e, s = q % RING;
            ok = mbar_wait_n(full0 + 8 * s, (q / RING) & 1, q == 0 ? a.first_limit : SPIN_LIMIT);
            if (!ok) break;
            ++consumed;
            fence_after_sync();
            const uint32_t sa = sbase + s * a.stage_bytes, sb = sa + A_TILE;
#pragma unroll
            for (int kk = 0; kk < NC / 16; ++kk)
                mma_16bit(acc, sdesc(sa + kk * 32), sdesc(sb + kk * 32), a.idesc, (e > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty0 + 8 * s);
        }
    }
    if (!ok) {
        for (int d = consumed; d < issued; ++d) {
            const uint32_t q = q0 + d;
            mbar_wait(full0 + 8 * (q % RING), (q / RING) & 1);
        }
    }
    mma_commit(done);
    q0 += 9;
    return ok;
}

// shared-memory overlay of the ring once a step's MMAs are complete
struct Overlay {
    float2 *W;       // [MAX_SITES][64][ldw]: the scaled stencil output w of each own site
    int ldw;         // n + 1 (padding against bank conflicts)
    float *Dhi;      // [64][ld]: accumulator rows 64..127 of one site while w is formed
    int ld;          // npad + 1
    uint8_t *tile;   // [MAX_SITES] x b_tile bytes: the own sites' packed images
    float2 *red;     // [RS][MMAX + 1][n] partial sums of the row slices
    float2 *coef;    // [MMAX][n] h (or y) coefficients
};

__host__ __device__ inline size_t overlay_bytes(int n, int npad, Overlay *o, uint8_t *base) {
    const int ldw = n + 1, ld = npad + 1;
    auto up = [](size_t v) { return (v + 127) & ~size_t(127); };
    size_t off = 0;
    const size_t w_off = off;
    off += up(sizeof(float2) * (size_t)MAX_SITES * NC * ldw);
    const size_t d_off = off;
    off += up(sizeof(float) * (size_t)NC * ld);
    const size_t tile_off = off;
    off += (size_t)MAX_SITES * npad * 128;
    const size_t red_off = off;
    off += sizeof(float2) * (size_t)THREADS * (MMAX + 1);  // >= (THREADS / n) slices x n columns, any n
    const size_t coef_off = off;
    off += sizeof(float2) * (size_t)MMAX * n;
    if (o) {
        o->W = reinterpret_cast<float2 *>(base + w_off);
        o->ldw = ldw;
        o->Dhi = reinterpret_cast<float *>(base + d_off);
        o->ld = ld;
        o->tile = base + tile_off;
        o->red = reinterpret_cast<float2 *>(base + red_off);
        o->coef = reinterpret_cast<float2 *>(base + coef_off);
    }
    return off;
}

__host__ __device__ inline size_t fused_smem_bytes(int n, int npad, uint32_t stage_bytes) {
    const size_t ring = (size_t)MAX_SITES * RING * stage_bytes;
    const size_t ov = overlay_bytes(n, npad, nullptr, nullptr);
    return (ring > ov ? ring : ov) + 1024;
}

template <int FMT>
__global__ void __launch_bounds__(THREADS, 1) k_coarsest_gmres(const FusedArgs a) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bars[2 * MAX_SITES * RING + 1];  // per own site: RING full, RING empty; then done
    __shared__ uint32_t tmem_base_sh;
    __shared__ int flag_sh, abort_sh;
    __shared__ double red_d[THREADS];
    __shared__ double eta_sh[64];
    // sig: scale of an image; inv: 1 / eta; cinv: 1 / (sig * eta), the per-RHS factor that turns
    // a site's accumulator (times its link scale) into A v_j
    __shared__ float sig_sh[64], inv_sh[64], cinv_sh[64];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cta = blockIdx.x;
    const int n = a.n, m = a.m;
    const int ns = (a.V - cta + a.G - 1) / a.G;  // this CTA's sites: cta + ls * G, ls < ns
    const int64_t F = (int64_t)a.V * NC * n;     // complex values per field
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(base);
    const uint32_t done = smem_u32(&bars[2 * MAX_SITES * RING]);
    // ring of own site ls: stages at ring_of(ls), barriers full_of(ls) / empty_of(ls)
    auto full_of = [&](int ls) { return smem_u32(&bars[2 * RING * ls]); };
    auto empty_of = [&](int ls) { return smem_u32(&bars[2 * RING * ls + RING]); };
    auto ring_of = [&](int ls) { return sbase + (uint32_t)(ls * RING) * a.stage_bytes; };
    Overlay ov;
    overlay_bytes(n, a.npad, &ov, base);
    const RowMap t(n);
    unsigned nbar = 0;
    uint32_t q0 = 0;
    auto site_of = [&](int ls) { return (int64_t)cta + (int64_t)ls * a.G; };
    auto row0_of = [&](int ls) { return site_of(ls) * NC * n; };
    auto tile_of = [&](int ls) { return ov.tile + (size_t)ls * a.b_tile; };
    auto Wrow = [&](int ls, int k) { return ov.W + ((size_t)ls * NC + k) * ov.ldw; };

    if (tid == 0) {
        for (int ls = 0; ls < MAX_SITES; ++ls)
            for (int s = 0; s < RING; ++s) {
                mbar_init(full_of(ls) + 8 * s, 1);
                mbar_init(empty_of(ls) + 8 * s, 1);
            }
        mbar_init(done, ns);  // one MMA commit per own site and step
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_base_sh), a.tmem_cols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_base_sh;

    // w of local site ls from its accumulator: Re w = sc (D[K][r] - D[64+K][n+r]), Im w = sc (D[64+K][r] +
    // D[K][n+r]) with sc = link scale * cinv[r].  Warp w reads tensor-memory lanes 32 (w % 4) .. + 31 and
    // every fourth 16-column chunk from chunk w / 4: the upper lanes first into Dhi, then the lower ones
    // combine.  Ends with a CTA barrier.
    auto stage_w = [&](int ls) {
        fence_after_sync();
        const int q = warp & 3, grp = warp >> 2;
        const float ls_scale = a.lscale[site_of(ls)];
        if (q >= 2) {
            const int K = 32 * (q - 2) + lane;
            for (int c0 = 16 * grp; c0 < a.npad; c0 += 16 * (THREADS / 128)) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ls * a.cols_site + c0), v);
#pragma unroll
                for (int i = 0; i < 16; ++i) ov.Dhi[K * ov.ld + c0 + i] = v[i];
            }
        }
        __syncthreads();
        if (q < 2) {
            const int K = 32 * q + lane;
            float2 *Wk = Wrow(ls, K);
            float *Wf = reinterpret_cast<float *>(Wk);
            for (int c0 = 16 * grp; c0 < a.npad; c0 += 16 * (THREADS / 128)) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ls * a.cols_site + c0), v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int c = c0 + i;
                    if (c < n) Wf[2 * c] = ls_scale * cinv_sh[c] * (v[i] - ov.Dhi[K * ov.ld + n + c]);
                    else if (c < 2 * n) Wf[2 * (c - n) + 1] = ls_scale * cinv_sh[c - n] * (ov.Dhi[K * ov.ld + c - n] + v[i]);
                }
            }
        }
        fence_before_sync();
        __syncthreads();
    };
    // the packed tile of local site ls -> its image in global memory (after the tile is complete)
    auto tile_out = [&](int ls) {
        uint4 *dst = reinterpret_cast<uint4 *>(a.img + (size_t)site_of(ls) * a.b_tile);
        const uint4 *src = reinterpret_cast<const uint4 *>(tile_of(ls));
        for (int i = tid; i < a.npad * 8; i += THREADS) dst[i] = src[i];
    };
    auto tiles_zero = [&]() {
        uint4 *t4 = reinterpret_cast<uint4 *>(ov.tile);
        for (int i = tid; i < ns * a.npad * 8; i += THREADS) t4[i] = make_uint4(0, 0, 0, 0);
    };
    auto pack = [&](int ls, int k, int r, float re, float im) {
        *reinterpret_cast<uint16_t *>(tile_of(ls) + sw128_offset(r, k)) = to16<FMT>(re);
        *reinterpret_cast<uint16_t *>(tile_of(ls) + sw128_offset(n + r, k)) = to16<FMT>(im);
    };
    // per-CTA norm partial: the row slices' sums in slice order
    auto norm_partial_out = [&](float un) {
        if (t.active) ov.red[t.sub * n + t.r] = make_float2(un, 0.f);
        __syncthreads();
        if (tid < n) {
            double s = 0.0;
            for (int q = 0; q < t.RS; ++q) s += (double)ov.red[q * n + tid].x;
            a.npart[(int64_t)cta * n + tid] = s;
        }
    };
    bool ok = true;

    // ---- prologue: V_0 = b (own rows), ||b||^2 partials; then the images of b scaled by 256 / ||b||
    {
        float acc = 0.f;
        if (t.active)
            for (int ls = 0; ls < ns; ++ls)
#pragma unroll 4
                for (int k = t.sub; k < NC; k += t.RS) {
                    const int64_t e = row0_of(ls) + (int64_t)k * n + t.r;
                    const float2 v = a.b[e];
                    a.Vb[e] = v;
                    acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
                }
        norm_partial_out(acc);
    }
    ok = grid_barrier(a, nbar, &flag_sh);
    if (ok) {
        reduce_norms(a, red_d, eta_sh);
        if (tid < n) sig_sh[tid] = eta_sh[tid] > 0.0 ? (float)(IMG_BOUND / eta_sh[tid]) : 1.f;
        tiles_zero();
        __syncthreads();
        if (t.active)
            for (int ls = 0; ls < ns; ++ls)
#pragma unroll 4
                for (int k = t.sub; k < NC; k += t.RS) {
                    const float2 v = a.Vb[row0_of(ls) + (int64_t)k * n + t.r];
                    const float sc = sig_sh[t.r];
                    pack(ls, k, t.r, v.x * sc, v.y * sc);
                }
        __syncthreads();
        for (int ls = 0; ls < ns; ++ls) tile_out(ls);
        if (cta == 0 && tid < n) a.sig[tid] = sig_sh[tid];
        fence_proxy_async_global();
        ok = grid_barrier(a, nbar, &flag_sh);
    }

    // ---- Arnoldi steps
    for (int j = 0; ok && j < m; ++j) {
        // (S) eta_j = ||u_j||; the per-RHS scalars of this step
        reduce_norms(a, red_d, eta_sh);
        if (tid < n) {
            const double eta = eta_sh[tid];
            const float sg = a.sig[tid];
            sig_sh[tid] = sg;
            inv_sh[tid] = eta > 0.0 ? (float)(1.0 / eta) : 0.f;
            cinv_sh[tid] = eta > 0.0 ? (float)(1.0 / ((double)sg * eta)) : 0.f;
        }
        __syncthreads();
        // (1) threads 0 and 64 stream the stencils of the first and the second own site through their
        // rings and the tensor cores; meanwhile thread 32 folds column j - 1 into the owned columns'
        // Givens state (h_{j,j-1} = eta_j) and every thread normalises its rows of v_j = u_j / eta_j
        if (tid == 0 || (tid == 64 && ns > 1)) {
            const int ls = tid == 0 ? 0 : 1;
            fence_proxy_async_global();  // the neighbours' images were written through the generic proxy
            if (!stencil_issue(a, site_of(ls), ring_of(ls), full_of(ls), empty_of(ls), done,
                               tmem + (uint32_t)(ls * a.cols_site), q0)) {
                record_error(a);
                abort_sh = 1;
            }
        } else if (tid == 32) {
            for (int r = cta; r < n; r += a.G) {
                if (j == 0) {
                    double2 *g = a.g + (int64_t)r * (m + 1);
                    g[0] = make_double2(eta_sh[r], 0.0);
                    for (int i = 1; i <= m; ++i) g[i] = make_double2(0.0, 0.0);
                } else {
                    givens_column(a, r, j - 1, eta_sh[r]);
                }
            }
        }
        {
            float2 *Vj = a.Vb + (int64_t)j * F;
            if (t.active)
                for (int ls = 0; ls < ns; ++ls)
#pragma unroll 4
                    for (int k = t.sub; k < NC; k += t.RS) {
                        const int64_t e = row0_of(ls) + (int64_t)k * n + t.r;
                        const float2 v = Vj[e];
                        Vj[e] = make_float2(v.x * inv_sh[t.r], v.y * inv_sh[t.r]);
                    }
        }
        __syncthreads();
        const bool mma_ok = mbar_wait(done, j & 1);
        // one decision for the whole CTA: a wait that expired in any thread stops it
        if (__syncthreads_or(abort_sh || !mma_ok)) {
            if (tid == 0) {
                record_error(a);
                mbar_wait(done, j & 1);  // one more bounded wait for issued MMAs before tensor memory is freed
            }
            ok = false;
            break;
        }
        for (int ls = 0; ls < ns; ++ls) stage_w(ls);
        // partial dots <v_i, w> (i <= j) and ||w||^2 over the own rows
        {
            float2 acc[MMAX];
#pragma unroll
            for (int i = 0; i < MMAX; ++i) acc[i] = make_float2(0.f, 0.f);
            float wn = 0.f;
            if (t.active)
                for (int ls = 0; ls < ns; ++ls)
#pragma unroll 4
                    for (int k = t.sub; k < NC; k += t.RS) {
                        const float2 w = Wrow(ls, k)[t.r];
                        wn = fmaf(w.x, w.x, fmaf(w.y, w.y, wn));
                        const int64_t e = row0_of(ls) + (int64_t)k * n + t.r;
#pragma unroll
                        for (int i = 0; i < MMAX; ++i)
                            if (i <= j) {
                                const float2 v = a.Vb[(int64_t)i * F + e];
                                acc[i].x = fmaf(v.x, w.x, fmaf(v.y, w.y, acc[i].x));
                                acc[i].y = fmaf(v.x, w.y, fmaf(-v.y, w.x, acc[i].y));
                            }
                    }
            if (t.active) {
#pragma unroll
                for (int i = 0; i < MMAX; ++i)
                    if (i <= j) ov.red[(t.sub * (MMAX + 1) + i) * n + t.r] = acc[i];
                ov.red[(t.sub * (MMAX + 1) + j + 1) * n + t.r] = make_float2(wn, 0.f);
            }
            __syncthreads();
            for (int e = tid; e < (j + 2) * n; e += THREADS) {
                const int i = e / n, r = e - i * n;
                double sx = 0.0, sy = 0.0;
                for (int q = 0; q < t.RS; ++q) {
                    const float2 p = ov.red[(q * (MMAX + 1) + i) * n + r];
                    sx += (double)p.x;
                    sy += (double)p.y;
                }
                a.part[((int64_t)cta * (m + 1) + i) * n + r] = make_double2(sx, sy);
            }
        }
        if (!(ok = grid_barrier(a, nbar, &flag_sh))) break;

        // (2) owners: h_{i,j} = sum over CTAs (i <= j), and the next image scale 256 / ||w||
        for (int r = cta; r < n; r += a.G) {
            for (int i0 = 0; i0 < j + 2; i0 += THREADS / 32) {
                const int i = i0 + warp, sub = lane;  // one warp per Hessenberg entry
                double sx = 0.0, sy = 0.0;
                if (i < j + 2)
#pragma unroll 8
                    for (int c = sub; c < a.G; c += 32) {
                        const double2 p = a.part[((int64_t)c * (m + 1) + i) * n + r];
                        sx += p.x;
                        sy += p.y;
                    }
                for (int o = 16; o > 0; o >>= 1) {
                    sx += __shfl_down_sync(0xffffffffu, sx, o);
                    sy += __shfl_down_sync(0xffffffffu, sy, o);
                }
                if (sub == 0 && i < j + 2) {
                    if (i <= j) a.hcol[(int64_t)i * n + r] = make_double2(sx, sy);
                    else a.sig[r] = sx > 0.0 ? (float)(IMG_BOUND / sqrt(sx)) : 1.f;
                }
            }
        }
        if (!(ok = grid_barrier(a, nbar, &flag_sh))) break;

        // (3) u_{j+1} = w - sum_i h_{i,j} v_i on own rows, the images of the own sites, ||u||^2 partials
        for (int e = tid; e < (j + 1) * n; e += THREADS) {
            const double2 h = a.hcol[e];
            ov.coef[e] = make_float2((float)h.x, (float)h.y);
        }
        if (tid < n) sig_sh[tid] = a.sig[tid];  // sigma_{j+1}
        tiles_zero();
        __syncthreads();
        {
            float un = 0.f;
            float2 *U = a.Vb + (int64_t)(j + 1) * F;
            if (t.active) {
                const float si = sig_sh[t.r];
                for (int ls = 0; ls < ns; ++ls)
#pragma unroll 4
                    for (int k = t.sub; k < NC; k += t.RS) {
                        const float2 w = Wrow(ls, k)[t.r];
                        float ur = w.x, ui = w.y;
                        const int64_t e = row0_of(ls) + (int64_t)k * n + t.r;
#pragma unroll
                        for (int i = 0; i < MMAX; ++i)
                            if (i <= j) {
                                const float2 v = a.Vb[(int64_t)i * F + e];
                                const float2 h = ov.coef[i * n + t.r];
                                ur = fmaf(-h.x, v.x, fmaf(h.y, v.y, ur));
                                ui = fmaf(-h.x, v.y, fmaf(-h.y, v.x, ui));
                            }
                        U[e] = make_float2(ur, ui);
                        un = fmaf(ur, ur, fmaf(ui, ui, un));
                        pack(ls, k, t.r, ur * si, ui * si);
                    }
            }
            __syncthreads();
            for (int ls = 0; ls < ns; ++ls) tile_out(ls);
            norm_partial_out(un);
            fence_proxy_async_global();
        }
        if (!(ok = grid_barrier(a, nbar, &flag_sh))) break;
    }

    // ---- fold the last column, y = R^-1 g (owners), x = sum_i y_i v_i on own rows
    if (ok) {
        reduce_norms(a, red_d, eta_sh);
        if (tid == 0)
            for (int r = cta; r < n; r += a.G) {
                givens_column(a, r, m - 1, eta_sh[r]);
                back_substitute(a, r);
            }
        ok = grid_barrier(a, nbar, &flag_sh);
    }
    if (ok) {
        for (int e = tid; e < m * n; e += THREADS) {
            const double2 yv = a.y[e];
            ov.coef[e] = make_float2((float)yv.x, (float)yv.y);
        }
        __syncthreads();
        if (t.active)
            for (int ls = 0; ls < ns; ++ls)
#pragma unroll 4
                for (int k = t.sub; k < NC; k += t.RS) {
                    const int64_t e = row0_of(ls) + (int64_t)k * n + t.r;
                    float xr = 0.f, xi = 0.f;
                    for (int i = 0; i < m; ++i) {
                        const float2 v = a.Vb[(int64_t)i * F + e];
                        const float2 c = ov.coef[i * n + t.r];
                        xr = fmaf(c.x, v.x, fmaf(-c.y, v.y, xr));
                        xi = fmaf(c.x, v.y, fmaf(c.y, v.x, xi));
                    }
                    a.x[e] = make_float2(xr, xi);
                }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

}  // namespace

size_t CoarsestFused::smem_bytes(int n) {
    const int npad = npad_of(n);
    const uint32_t b_tile = (uint32_t)npad * 128u;
    const uint32_t stage = A_TILE + ((b_tile + 1023u) & ~1023u);
    return fused_smem_bytes(n, npad, stage);
}

int CoarsestFused::resident_ctas(const Level &c, int nmax, int device) {
    if (!c.Abf.ptr || c.dof != NC || nmax < 1 || nmax > 64) return 0;
    int coop = 0;
    MRHS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    if (!coop) return 0;
    const void *kern = c.tc_fmt == MRHS_FP16 ? reinterpret_cast<const void *>(k_coarsest_gmres<0>)
                                             : reinterpret_cast<const void *>(k_coarsest_gmres<1>);
    // the attribute allows the largest size of any hierarchy; a launch takes its own
    MRHS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(64)));
    // a kernel that allocates tensor memory counts as one CTA per SM for residency (the
    // occupancy calculator and the cooperative launch check)
    int per_sm = 0;
    MRHS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem_bytes(nmax)));
    return per_sm * sm_count(device);
}

int CoarsestFused::max_sites_per_cta(int nmax) {
    const int per = 512 / (int)tmem_cols_for(npad_of(nmax));  // one accumulator per site in 512 columns
    return per < MAX_SITES ? per : MAX_SITES;
}

bool CoarsestFused::supported(const Level &c, int nmax, int m, int device) {
    if (nmax < 1 || nmax > 64 || m < 1 || m > MMAX) return false;
    return (int64_t)resident_ctas(c, nmax, device) * max_sites_per_cta(nmax) >= c.V;
}

void CoarsestFused::init(const Level &c, int m_, int nmax_, int device) {
    m = m_;
    nmax = nmax_;
    const int cap = resident_ctas(c, nmax, device);
    S = (int)((c.V + cap - 1) / cap);       // sites per CTA
    G = (int)((c.V + S - 1) / S);           // CTAs, each with S sites but the last ones
    part.alloc(sizeof(double2) * (size_t)G * (m + 1) * nmax);
    npart.alloc(sizeof(double) * (size_t)G * nmax);
    hcol.alloc(sizeof(double2) * (size_t)(m + 1) * nmax);
    sig.alloc(sizeof(float) * (size_t)nmax);
    R.alloc(sizeof(double2) * (size_t)nmax * (m + 1) * m);
    cs.alloc(sizeof(double) * (size_t)nmax * m);
    sn.alloc(sizeof(double2) * (size_t)nmax * m);
    g.alloc(sizeof(double2) * (size_t)nmax * (m + 1));
    y.alloc(sizeof(double2) * (size_t)m * nmax);
    sync.alloc(sizeof(unsigned) * 2);
}

void CoarsestFused::solve(const Level &c, float2 *Vbasis, const float2 *b, float2 *x, int n, cudaStream_t s) {
    if (n < 1 || n > nmax) fail(MRHS_ERR_INVALID, "fused coarsest solve: RHS count above the workspace");
    FusedArgs a;
    for (int mu = 0; mu < 4; ++mu) a.L[mu] = c.L[mu];
    a.G = G;
    a.V = (int)c.V;
    a.S = S;
    a.n = n;
    a.npad = npad_of(n);
    a.m = m;
    a.idesc = idesc_16bit(MROWS, a.npad, c.tc_fmt == MRHS_FP16 ? 0u : 1u);
    a.cols_site = (int)tmem_cols_for(a.npad);
    a.tmem_cols = 32;  // the allocation: a power of two >= 32, at most 512 (S is bounded in supported)
    while (a.tmem_cols < (uint32_t)(S * a.cols_site)) a.tmem_cols *= 2;
    a.b_tile = (uint32_t)a.npad * 128u;
    a.stage_bytes = A_TILE + ((a.b_tile + 1023u) & ~1023u);
    a.Abf = c.Abf.as<uint8_t>();
    a.lscale = c.LinkScale.as<float>();
    a.img = c.PhiBf.as<uint8_t>();
    a.b = b;
    a.x = x;
    a.Vb = Vbasis;
    a.part = part.as<double2>();
    a.npart = npart.as<double>();
    a.hcol = hcol.as<double2>();
    a.sig = sig.as<float>();
    a.R = R.as<double2>();
    a.cs = cs.as<double>();
    a.sn = sn.as<double2>();
    a.g = g.as<double2>();
    a.y = y.as<double2>();
    a.sync = sync.as<unsigned>();
    a.err = c.TcErr.as<int>();
    a.first_limit = tc_first_wait_limit(s);
    zero_on_sms(sync.ptr, sizeof(unsigned) * 2, s);
    const size_t smem = smem_bytes(nmax);  // covers every n <= nmax (the sizes grow with n)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MRHS_TIMED("k_coarsest_gmres", s);
    if (c.tc_fmt == MRHS_FP16) MRHS_CUDA(cudaLaunchKernelEx(&cfg, k_coarsest_gmres<0>, a));
    else MRHS_CUDA(cudaLaunchKernelEx(&cfg, k_coarsest_gmres<1>, a));
    MRHS_LAUNCHED("k_coarsest_gmres");
}

}  // namespace mrhs
