// Warp-specialised tcgen05 GEMM engine of the mixed-precision path.
//
// One CTA = 10 warps:
//   warp 0      TMA producer (one elected lane) filling a ring of smem stages
//   warp 1      MMA issuer (one elected lane) + TMEM owner
//   warps 2..9  epilogue: TMEM -> registers -> fused math -> global
// Accumulators live in TMEM, double buffered, so the epilogue of one tile
// overlaps the MMAs of the next.
// The forward modes also run on CTA pairs (clusters of two, tc_engine_pair):
// the two CTAs take consecutive 128-point blocks of the same 128 output
// features, each loads its own A rows and HALF of the weight rows, and the
// even CTA issues 256-row MMAs (cta_group::2) over both CTAs' shared memory,
// so each SM receives 24 KB instead of 32 KB per 64-deep K block of a tile.  A CTA walks a short list of output tiles
// (e.g. the Taylor columns s of one point block) so that per-(point, feature)
// state such as tanh'(a_0) or the running sum of squared tangents stays in
// registers across tiles.
//
// Modes (template parameter):
//   FWD_VALUE   value rows of a layer: a_0 = acc + b, y_0 = tanh(a_0)
//   FWD_TANLAP  tangent rows y_i = s1 a_i and the Laplacian pre-activation,
//               partial sums of a_i^2 over the CTA's chunk of columns (Eq. 6)
//   BWD_LAP     adjoint of the Laplacian rows: abar_D = s1 ybar_D
//   BWD_TAN     adjoint of tangent rows: abar_i = s1 ybar_i - 4 y_0 y_i ybar_D
//   BWD_VALUE   adjoint of value rows (uses the tangent cross sums)
//   GRAM        C = X^T Y over a chunk of rows (factor Grams, weight gradient)
//   JDOT        residual Jacobian-vector products of a layer (KFAC*): the
//               rows of T^ V~^T (V~ = (V b_v) a direction shaped like W~)
//               dotted with the stored adjoint rows g of the same Taylor
//               column and point, summed over the CTA's columns:
//               <dr_n/dW~_l, V~> = sum_s g_{n,s}^T V~ T^_{n,s} (Sec. 3.2)
#pragma once
#include "tc_common.cuh"
#include "group.cuh"

namespace tck {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int NUM_THREADS = 320;
constexpr int EPI_WARPS = 8;

enum Mode { FWD_VALUE = 0, FWD_TANLAP = 1, BWD_LAP = 2, BWD_TAN = 3, BWD_VALUE = 4, GRAM = 5, JDOT = 6 };

struct Args {
    CUtensorMap a0, a1, b0, b1;     // operand maps; a1/b1 carry the low BF16 halves
    int N_pad, N, S;                // pass geometry (points padded to 128)
    int k_steps;                    // contraction length / 64 (FWD/BWD modes)
    int n_out;                      // real output features
    int hp_out;                     // row stride of the outputs (elements)
    const float* chw;               // weights of the tangent columns in the second-order column (d)
    int split_time;                 // heat: the time tangent row (s = 1) is split-BF16 too
    int chunk_len, n_chunks;        // tangent-column chunking over blockIdx.z
    // GRAM
    int P, Q, rows, row_chunk, sym, q_tiles;
    // epilogue data
    __nv_bfloat16* out_hi;          // FWD: T^{(l)} hi; BWD: g^{(l-1)}
    __nv_bfloat16* out_lo;          // FWD: lo block (value, Laplacian)
    __nv_bfloat16* out_gr;          // BWD: r_n * g^{(l-1)}
    const float* bias;              // FWD_VALUE
    float* A0;                      // pre-activation a_0          (N_pad x hp_out)
    float* AD;                      // pre-activation a_Delta
    float* SSQ;                     // sum of squared tangents
    float* YD;                      // ybar_Delta (BWD)
    float* part;                    // chunk partials / Gram partials
    const __nv_bfloat16* ytan;      // BWD_TAN: T^{(l-1)} (y_i)
    const __nv_bfloat16* g_hi;      // JDOT: adjoint rows g^{(l)} (high half)
    const __nv_bfloat16* g_lo;      // JDOT: their low halves (split-BF16 everywhere), or nullptr
    const double* r;                // residuals (BWD: for r_n g)
    int* status;
    // split-BF16 on every row (tc_engine<MODE, true>): low halves laid out like the high ones
    int split_all;
    __nv_bfloat16* out_gr_lo;       // BWD: low half of r_n * g
    const __nv_bfloat16* ytan_lo;   // BWD_TAN: low half of y_i
};

template <int MODE, bool SPLIT = false, bool PAIR = false>
struct Cfg {
    static_assert(!PAIR || MODE == FWD_VALUE || MODE == FWD_TANLAP, "CTA pairs: forward modes only");
    static constexpr bool MN = (MODE == GRAM);
    static constexpr int BN = MN ? 256 : 128;
    static constexpr int BN_CTA = PAIR ? BN / 2 : BN;     // weight rows one CTA loads
    // Two-slot stages: a stage holds two A and two B boxes (each one 64-wide K
    // block, one 128-byte-swizzled TMA box).  A tile with a single product per
    // K block fills the slots with two consecutive K blocks (half the barrier
    // round trips for the same bytes in flight: measured 16 % faster for the
    // forward modes); a tile with several products per K block (the split-BF16
    // terms hi*hi + hi*lo + lo*hi) fills them with the two A and the two B
    // operands of ONE K block and issues every product from them, so each
    // operand crosses L2 -> SM once per K block instead of once per product.
    // The forward and JDOT modes always use two slots; the
    // adjoint modes only when every row is split (one slot and six stages
    // otherwise); the Gram keeps one slot.
    static constexpr bool FUSED =
        (MODE == FWD_VALUE || MODE == FWD_TANLAP || MODE == JDOT) ||
        (SPLIT && (MODE == BWD_LAP || MODE == BWD_TAN || MODE == BWD_VALUE));
    static constexpr int SLOTS = FUSED ? 2 : 1;
    static constexpr int STAGES = MN ? 4 : (PAIR ? 4 : (FUSED ? 3 : 6));
    static constexpr int SLOT_A = BM * BK * 2;
    static constexpr int SLOT_B = BN_CTA * BK * 2;
    static constexpr int A_BYTES = SLOTS * SLOT_A;
    static constexpr int B_BYTES = SLOTS * SLOT_B;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
    static constexpr int TMEM_COLS = MN ? 256 : 2 * BN;
    static constexpr int NBUF = MN ? 1 : 2;
    static constexpr uint32_t IDESC = tc::idesc_bf16(PAIR ? 2 * BM : BM, BN, MN ? 1 : 0, MN ? 1 : 0);
    // bytes one stage's full barrier waits for (a pair's even CTA counts both CTAs' loads)
    static constexpr uint32_t TX_BYTES = PAIR ? 2 * STAGE_BYTES : STAGE_BYTES;
};

// Number of accumulation terms of tile s (split-BF16 on value/Laplacian rows).
template <int MODE>
KFAC_DEV int n_terms(int s, int S, int split_time, int split_all) {
    if (MODE == FWD_VALUE) return 3;
    if (split_all) return 3;                              // hi x hi + hi x lo + lo x hi everywhere
    if (MODE == FWD_TANLAP) return (s == S - 1 || (split_time && s == 1)) ? 3 : 1;
    if (MODE == JDOT) return (s == 0 || s == S - 1 || (split_time && s == 1)) ? 3 : 1;
    return 1;
}

// Block of the low-half tensor holding row block s: value 0, Laplacian 1, time 2.
KFAC_DEV int lo_block(int s, int S) { return s == 0 ? 0 : (s == S - 1 ? 1 : 2); }

template <int MODE>
KFAC_DEV void tile_range(const Args& a, uint3 vb, int& s_begin, int& s_end) {
    if (MODE == FWD_VALUE || MODE == BWD_VALUE || MODE == GRAM) { s_begin = 0; s_end = 1; return; }
    if (MODE == BWD_LAP) { s_begin = a.S - 1; s_end = a.S; return; }
    if (MODE == JDOT) {       // every Taylor column, value row block included
        s_begin = vb.z * a.chunk_len;
        s_end = min(a.S, s_begin + a.chunk_len);
        return;
    }
    int last = (MODE == FWD_TANLAP) ? a.S : a.S - 1;   // FWD covers the Laplacian tile too
    s_begin = 1 + vb.z * a.chunk_len;
    s_end = min(last, s_begin + a.chunk_len);
}

KFAC_DEV float bf_round_lo(float v, __nv_bfloat16& hi) {
    hi = __float2bfloat16_rn(v);
    return v - __bfloat162float(hi);
}

KFAC_DEV void store16_bf16(__nv_bfloat16* dst, const float* v) {
    __align__(16) __nv_bfloat162 t[8];
#pragma unroll
    for (int i = 0; i < 8; i++) t[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    uint4* d = reinterpret_cast<uint4*>(dst);
    const uint4* s = reinterpret_cast<const uint4*>(t);
    d[0] = s[0];
    d[1] = s[1];
}

KFAC_DEV void load16_bf16(const __nv_bfloat16* src, float* v) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    __align__(16) uint4 t[2];
    t[0] = s[0];
    t[1] = s[1];
    const __nv_bfloat162* p = reinterpret_cast<const __nv_bfloat162*>(t);
#pragma unroll
    for (int i = 0; i < 8; i++) {
        float2 f = __bfloat1622float2(p[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

KFAC_DEV void store16_f32(float* dst, const float* v) {
    float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int i = 0; i < 4; i++) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

KFAC_DEV void load16_f32(const float* src, float* v) {
    const float4* s = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float4 f = s[i];
        v[4 * i] = f.x; v[4 * i + 1] = f.y; v[4 * i + 2] = f.z; v[4 * i + 3] = f.w;
    }
}

// ---------------------------------------------------------------------------
// SPLIT (split-BF16 on every row, Args::split_all) is a template parameter so
// that the plain instantiations keep their register budget.
// The engine's work for one CTA: vb / vg stand for blockIdx / gridDim of the
// launch the CTA belongs to (its own, or its member's in a grouped launch).
// Inlined into both the solo and the grouped kernel.  Their translation unit
// (tc_engine.cu) is compiled without floating-point contraction: every FMA is
// an explicit fmaf, so the two copies round alike and a member of a grouped
// launch computes exactly what its own launch computes.
//
// PAIR: the CTA is one of a cluster of two (tc_engine_pair).  vb.x is then
// 2 j + r for feature tile j and rank r in the pair, vb.y the pair of point
// blocks (2 vb.y + r), so that, as in the single-CTA grid, the CTAs that run
// together share their point block's rows (in L2) across the feature tiles.  The
// even CTA's full barriers count both CTAs' TMA bytes and its MMA thread
// issues the pair MMAs; their commits arrive on the stage and accumulator
// barriers of both CTAs; both CTAs' epilogue warps arrive on the even CTA's
// accumulator-empty barriers.  The pair synchronises (barrier.cluster) after
// the set-up and before leaving, so that neither CTA leaves while the other
// may still touch its shared memory.
template <int MODE, bool SPLIT, bool PAIR = false>
KFAC_DEV void engine_body(const Args& a, const uint3 vb, const uint3 vg) {
    using C = Cfg<MODE, SPLIT, PAIR>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[C::STAGES], empty_bar[C::STAGES];
    __shared__ uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t rank = PAIR ? tc::cluster_ctarank() : 0u;

    // ---- tile geometry ----------------------------------------------------
    int p0, j0, s_begin, s_end, k_begin = 0, k_steps;
    if (MODE == GRAM) {
        // vb.x enumerates the (p, q) output tiles, symmetric ones only
        // when they touch the upper triangle; vb.y is the row chunk.
        int t = vb.x, pb = 0, qb = 0, cnt = 0;
        int p_tiles = (a.P + BM - 1) / BM;
        for (pb = 0; pb < p_tiles; pb++) {
            int q_first = a.sym ? (pb * BM) / C::BN : 0;
            int n = a.q_tiles - q_first;
            if (t < cnt + n) { qb = q_first + (t - cnt); break; }
            cnt += n;
        }
        p0 = pb * BM;
        j0 = qb * C::BN;
        k_begin = vb.y * a.row_chunk;
        int k_end = min(a.rows, k_begin + a.row_chunk);
        k_steps = (k_end - k_begin + BK - 1) / BK;
        s_begin = 0; s_end = 1;
    } else {
        j0 = (PAIR ? (vb.x >> 1) : vb.x) * C::BN;
        p0 = (PAIR ? 2 * vb.y + (vb.x & 1) : vb.y) * BM;
        k_steps = a.k_steps;                              // 64-wide K blocks (one-slot modes)
        tile_range<MODE>(a, vb, s_begin, s_end);
    }
    const int n_tiles = max(0, s_end - s_begin);

    if (threadIdx.x == 0) {
        for (int i = 0; i < C::STAGES; i++) { tc::mbar_init(&full_bar[i], 1); tc::mbar_init(&empty_bar[i], 1); }
        for (int i = 0; i < 2; i++) {
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_empty[i], PAIR ? 2 * EPI_WARPS : EPI_WARPS);
        }
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        tc::prefetch_tmap(&a.a0); tc::prefetch_tmap(&a.b0);
        if (MODE == FWD_VALUE || MODE == FWD_TANLAP || MODE == JDOT || SPLIT) {
            tc::prefetch_tmap(&a.a1);
            tc::prefetch_tmap(&a.b1);
        }
    }
    if (warp == 1) {
        if (PAIR) { tc::tmem_alloc_pair(&tmem_base, C::TMEM_COLS); tc::tmem_relinquish_pair(); }
        else { tc::tmem_alloc(&tmem_base, C::TMEM_COLS); tc::tmem_relinquish(); }
    }
    tc::tc_fence_before();
    if (PAIR) tc::cluster_sync();
    else __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = tmem_base;

    if (warp == 0) {
        // ============================ TMA producer ==========================
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            for (int ti = 0; ti < n_tiles && !abort_flag; ti++) {
                const int s = s_begin + ti;
                const int terms = SPLIT ? n_terms<MODE>(s, a.S, a.split_time, 1) : n_terms<MODE>(s, a.S, a.split_time, 0);
                if constexpr (C::FUSED) {
                    // rows of the second A operand: the low half, laid out like the high
                    // half when every row is split, else in its value / Laplacian / time block
                    const int arow = s * a.N_pad + p0;
                    const int arow1 = SPLIT ? arow : (lo_block(s, a.S) * a.N_pad + p0);
                    const bool fuse = terms > 1;
                    const int nst = fuse ? a.k_steps : (a.k_steps + 1) / 2;
                    // weight rows of this CTA (a pair's CTAs load one half each)
                    const int brow = j0 + (int)rank * C::BN_CTA;
                    for (int k = 0; k < nst; k++) {
                        if (!tc::mbar_wait(&empty_bar[stage], phase ^ 1)) { abort_flag = 1; break; }
                        unsigned char* sa = smem + stage * C::STAGE_BYTES;
                        unsigned char* sb = sa + C::A_BYTES;
                        // the odd CTA of a pair signals the even CTA's full barrier, armed there
                        const uint32_t fb = (PAIR && rank != 0) ? tc::mapa_shared(&full_bar[stage], 0) : 0u;
                        auto load = [&](void* dst, const CUtensorMap* m, int x, int y) {
                            if (PAIR && rank != 0) tc::tma_load_2d_pair(dst, m, fb, x, y);
                            else tc::tma_load_2d(dst, m, &full_bar[stage], x, y);
                        };
                        if (!PAIR || rank == 0) tc::mbar_arrive_expect_tx(&full_bar[stage], C::TX_BYTES);
                        if (fuse) {      // a0, a1, b0, b1 of K block k
                            const int kx = k * BK;
                            load(sa, &a.a0, kx, arow);
                            load(sa + C::SLOT_A, &a.a1, kx, arow1);
                            load(sb, &a.b0, kx, brow);
                            load(sb + C::SLOT_B, &a.b1, kx, brow);
                        } else {         // K blocks 2k and 2k+1 (blocks past K read zeros)
#pragma unroll
                            for (int u = 0; u < 2; u++) {
                                const int kx = (2 * k + u) * BK;
                                load(sa + u * C::SLOT_A, &a.a0, kx, arow);
                                load(sb + u * C::SLOT_B, &a.b0, kx, brow);
                            }
                        }
                        if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                    }
                } else {
                    for (int term = 0; term < terms && !abort_flag; term++) {
                        for (int k = 0; k < k_steps; k++) {
                            if (!tc::mbar_wait(&empty_bar[stage], phase ^ 1)) { abort_flag = 1; break; }
                            unsigned char* sa = smem + stage * C::STAGE_BYTES;
                            unsigned char* sb = sa + C::A_BYTES;
                            tc::mbar_arrive_expect_tx(&full_bar[stage], C::STAGE_BYTES);
                            if (MODE == GRAM) {
                                // terms: X_hi^T Y_hi, X_hi^T Y_lo, X_lo^T Y_hi
                                const int row = k_begin + k * BK;
                                const CUtensorMap* am = (term == 2) ? &a.a1 : &a.a0;
                                const CUtensorMap* bm = (term == 1) ? &a.b1 : &a.b0;
                                tc::tma_load_2d(sa, am, &full_bar[stage], p0, row);
                                tc::tma_load_2d(sa + 8192, am, &full_bar[stage], p0 + 64, row);
#pragma unroll
                                for (int b = 0; b < C::BN / 64; b++)
                                    tc::tma_load_2d(sb + 8192 * b, bm, &full_bar[stage], j0 + 64 * b, row);
                            } else {
                                // one slot: term 0 hi x hi, term 1 hi x W_lo, term 2 lo x W_hi
                                const CUtensorMap* am = (term == 2) ? &a.a1 : &a.a0;
                                const CUtensorMap* bm = (term == 1) ? &a.b1 : &a.b0;
                                int arow;
                                if constexpr (SPLIT) arow = s * a.N_pad + p0;   // low halves laid out like the high
                                else arow = (term == 2) ? (lo_block(s, a.S) * a.N_pad + p0) : (s * a.N_pad + p0);
                                const int kx = k * BK;
                                tc::tma_load_2d(sa, am, &full_bar[stage], kx, arow);
                                tc::tma_load_2d(sb, bm, &full_bar[stage], kx, j0);
                            }
                            if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                        }
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ============================ MMA issuer ============================
        // (a pair's MMAs are issued by the even CTA alone)
        if (lane == 0 && (!PAIR || rank == 0)) {
            int stage = 0;
            uint32_t phase = 0;
            for (int ti = 0; ti < n_tiles && !abort_flag; ti++) {
                const int s = s_begin + ti;
                const int buf = ti % C::NBUF;
                const uint32_t use = (uint32_t)(ti / C::NBUF);
                if (!tc::mbar_wait(&acc_empty[buf], (use & 1) ^ 1)) { abort_flag = 1; break; }
                tc::tc_fence_after();
                const uint32_t dcol = tbase + (uint32_t)(buf * C::BN);
                const int terms = SPLIT ? n_terms<MODE>(s, a.S, a.split_time, 1) : n_terms<MODE>(s, a.S, a.split_time, 0);
                bool first = true;
                if constexpr (C::FUSED) {
                    const bool fuse = terms > 1;
                    const int nst = fuse ? a.k_steps : (a.k_steps + 1) / 2;
                    for (int k = 0; k < nst; k++) {
                        if (!tc::mbar_wait(&full_bar[stage], phase)) { abort_flag = 1; break; }
                        tc::tc_fence_after();
                        const uint32_t sa = tc::smem_u32(smem + stage * C::STAGE_BYTES);
                        const uint32_t sb = sa + C::A_BYTES;
                        // (A slot, B slot) of each product: one K block per slot pair when
                        // not fused; hi*hi, hi*lo, lo*hi of one K block when fused
                        const int np = fuse ? 3 : 2;
#pragma unroll
                        for (int pi = 0; pi < 3; pi++) {
                            if (pi >= np) break;
                            const uint32_t ua = fuse ? (pi == 2 ? 1u : 0u) : pi;
                            const uint32_t ub = fuse ? (pi == 1 ? 1u : 0u) : pi;
#pragma unroll
                            for (int w = 0; w < BK / 16; w++) {
                                const uint64_t ad = tc::smem_desc(sa + ua * C::SLOT_A + w * 32, 16, 1024, tc::LAYOUT_SW128);
                                const uint64_t bd = tc::smem_desc(sb + ub * C::SLOT_B + w * 32, 16, 1024, tc::LAYOUT_SW128);
                                if (PAIR) tc::mma_bf16_pair(dcol, ad, bd, C::IDESC, first ? 0u : 1u);
                                else tc::mma_bf16(dcol, ad, bd, C::IDESC, first ? 0u : 1u);
                                first = false;
                            }
                        }
                        if (PAIR) tc::mma_commit_pair(&empty_bar[stage]);
                        else tc::mma_commit(&empty_bar[stage]);
                        if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                    }
                } else {
                    for (int term = 0; term < terms && !abort_flag; term++) {
                        for (int k = 0; k < k_steps; k++) {
                            if (!tc::mbar_wait(&full_bar[stage], phase)) { abort_flag = 1; break; }
                            tc::tc_fence_after();
                            const uint32_t sa = tc::smem_u32(smem + stage * C::STAGE_BYTES);
                            const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
                            for (int kk = 0; kk < BK / 16; kk++) {
                                uint64_t ad, bd;
                                if (C::MN) {
                                    ad = tc::smem_desc(sa + kk * 2048, 8192, 1024, tc::LAYOUT_SW128);
                                    bd = tc::smem_desc(sb + kk * 2048, 8192, 1024, tc::LAYOUT_SW128);
                                } else {
                                    ad = tc::smem_desc(sa + kk * 32, 16, 1024, tc::LAYOUT_SW128);
                                    bd = tc::smem_desc(sb + kk * 32, 16, 1024, tc::LAYOUT_SW128);
                                }
                                tc::mma_bf16(dcol, ad, bd, C::IDESC, first ? 0u : 1u);
                                first = false;
                            }
                            tc::mma_commit(&empty_bar[stage]);
                            if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                        }
                    }
                }
                if (PAIR) tc::mma_commit_pair(&acc_full[buf]);
                else tc::mma_commit(&acc_full[buf]);
            }
        }
    } else {
        // ============================ epilogue ==============================
        const int q = warp & 3;                          // TMEM lane quadrant of this warp
        const int half = (warp - 2) / 4;                 // column half
        const int r = q * 32 + lane;                     // row within the tile
        constexpr int CW = C::BN / 2;                    // columns per thread
        const int c0 = half * CW;
        const uint32_t lane_off = ((uint32_t)(q * 32)) << 16;
        const int n = p0 + r;                            // point (FWD/BWD)
        const long long hp = a.hp_out;
        // the odd CTA of a pair grid whose number of point blocks is odd: it
        // takes part in the pair's MMAs and barriers but touches no row
        const bool idle = PAIR && p0 >= a.N_pad;

        // per-thread state kept across the CTA's tiles
        constexpr bool STATE = (MODE == FWD_TANLAP || MODE == BWD_TAN);
        float st1[STATE ? CW : 1];
        float st2[STATE ? CW : 1];
        __nv_bfloat16 stq[(MODE == BWD_TAN) ? CW : 1];
        float jacc = 0.f;                                // JDOT: this thread's partial dot
        if (STATE) {
#pragma unroll
            for (int c = 0; c < CW; c += 16) {
                if (idle || j0 + c0 + c >= a.hp_out) {
#pragma unroll
                    for (int i = 0; i < 16; i++) { st1[c + i] = 0.f; st2[c + i] = 0.f; }
                    continue;
                }
                float a0v[16];
                load16_f32(a.A0 + (long long)n * hp + j0 + c0 + c, a0v);
                float ydv[16];
                if (MODE == BWD_TAN) load16_f32(a.YD + (long long)n * hp + j0 + c0 + c, ydv);
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    float y0 = tanhf(a0v[i]);
                    st1[c + i] = 1.f - y0 * y0;
                    st2[c + i] = 0.f;
                    if (MODE == BWD_TAN) stq[c + i] = __float2bfloat16_rn(4.f * y0 * ydv[i]);
                }
            }
        }
        for (int ti = 0; ti < n_tiles; ti++) {
            const int s = s_begin + ti;
            const int buf = ti % C::NBUF;
            const uint32_t use = (uint32_t)(ti / C::NBUF);
            bool ok = tc::mbar_wait(&acc_full[buf], use & 1);
            if (!ok) { abort_flag = 1; break; }
            tc::tc_fence_after();
            const uint32_t tcol = tbase + lane_off + (uint32_t)(buf * C::BN + c0);
#pragma unroll
            for (int c = 0; c < CW; c += 16) {
                if (idle) continue;                          // uniform over the CTA
                float v[16];
                tc::tmem_ld16(tcol + c, v);
                tc::tmem_wait_ld();
                const int j = j0 + c0 + c;
                if (MODE == GRAM) {
                    const int p = p0 + r;
                    if (p < a.P) {
                        float* dst = a.part + ((long long)vb.y * a.P + p) * a.Q + j;
                        // float4 stores need 16-byte alignment: Q % 4 == 0
                        if (j + 16 <= a.Q && (a.Q & 3) == 0) store16_f32(dst, v);
                        else for (int i = 0; i < 16 && j + i < a.Q; i++) dst[i] = v[i];
                    }
                    continue;
                }
                if (j >= a.hp_out) continue;
                const bool live = (n < a.N);
                if (MODE == FWD_VALUE) {
                    float a0v[16], hi[16], lo[16];
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        bool valid = live && (j + i < a.n_out);
                        float z = valid ? v[i] + a.bias[j + i] : 0.f;
                        a0v[i] = z;
                        float y0 = valid ? tanhf(z) : 0.f;
                        __nv_bfloat16 h;
                        lo[i] = bf_round_lo(y0, h);
                        hi[i] = __bfloat162float(h);
                    }
                    store16_f32(a.A0 + (long long)n * hp + j, a0v);
                    store16_bf16(a.out_hi + (long long)n * hp + j, hi);
                    store16_bf16(a.out_lo + (long long)n * hp + j, lo);
                } else if (MODE == JDOT) {
                    // (T^ V~^T)_{row, j}, the bias of V~ on the value rows, times g_{row, j}
                    if (live) {
                        float gh[16], gl[16];
                        const long long o = ((long long)s * a.N_pad + n) * hp + j;
                        load16_bf16(a.g_hi + o, gh);
                        if (a.g_lo) load16_bf16(a.g_lo + o, gl);
#pragma unroll
                        for (int i = 0; i < 16; i++) {
                            const float pv = (s == 0) ? v[i] + a.bias[j + i] : v[i];
                            const float gv = a.g_lo ? gh[i] + gl[i] : gh[i];
                            jacc = fmaf(pv, gv, jacc);
                        }
                    }
                } else if (MODE == FWD_TANLAP) {
                    if (s == a.S - 1) {
                        store16_f32(a.AD + (long long)n * hp + j, v);
                    } else {
                        float y[16];
                        const float wc = a.chw[s - 1];
#pragma unroll
                        for (int i = 0; i < 16; i++) {
                            y[i] = st1[c + i] * v[i];
                            st2[c + i] = fmaf(wc * v[i], v[i], st2[c + i]);
                        }
                        if constexpr (SPLIT) {
                            float hi[16], lo[16];
#pragma unroll
                            for (int i = 0; i < 16; i++) {
                                __nv_bfloat16 hb;
                                lo[i] = bf_round_lo(y[i], hb);
                                hi[i] = __bfloat162float(hb);
                            }
                            store16_bf16(a.out_hi + ((long long)s * a.N_pad + n) * hp + j, hi);
                            store16_bf16(a.out_lo + ((long long)s * a.N_pad + n) * hp + j, lo);
                        } else if (a.split_time && s == 1) {
                            float hi[16], lo[16];
#pragma unroll
                            for (int i = 0; i < 16; i++) {
                                __nv_bfloat16 hb;
                                lo[i] = bf_round_lo(y[i], hb);
                                hi[i] = __bfloat162float(hb);
                            }
                            store16_bf16(a.out_hi + ((long long)s * a.N_pad + n) * hp + j, hi);
                            store16_bf16(a.out_lo + (2LL * a.N_pad + n) * hp + j, lo);
                        } else {
                            store16_bf16(a.out_hi + ((long long)s * a.N_pad + n) * hp + j, y);
                        }
                    }
                } else {
                    // backward modes: v = ybar (T^bar) of this row block
                    const float rn = live ? (a.r ? (float)a.r[n] : 1.f) : 0.f;   // r == nullptr: Gr = g
                    float ab[16], gr[16];
                    if (MODE == BWD_LAP) {
                        float a0v[16];
                        load16_f32(a.A0 + (long long)n * hp + j, a0v);
#pragma unroll
                        for (int i = 0; i < 16; i++) {
                            float y0 = tanhf(a0v[i]);
                            ab[i] = (1.f - y0 * y0) * v[i];
                        }
                        store16_f32(a.YD + (long long)n * hp + j, v);
                    } else if (MODE == BWD_TAN) {
                        float yi[16];
                        load16_bf16(a.ytan + ((long long)s * a.N_pad + n) * hp + j, yi);
                        const float wc = a.chw[s - 1];
                        if (SPLIT) {
                            // full-precision y_i and 4 y_0 ybar_D (reloaded: FP32 state for
                            // it would not fit the registers beside st1 and st2)
                            float yl[16], a0v[16], ydv[16];
                            load16_bf16(a.ytan_lo + ((long long)s * a.N_pad + n) * hp + j, yl);
                            load16_f32(a.A0 + (long long)n * hp + j, a0v);
                            load16_f32(a.YD + (long long)n * hp + j, ydv);
#pragma unroll
                            for (int i = 0; i < 16; i++) {
                                const float y = yi[i] + yl[i];
                                float t = st1[c + i] * v[i];
                                t -= wc * (4.f * tanhf(a0v[i]) * ydv[i]) * y;
                                ab[i] = t;
                                st2[c + i] = fmaf(y, v[i], st2[c + i]);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; i++) {
                                float t = st1[c + i] * v[i];
                                t -= wc * __bfloat162float(stq[c + i]) * yi[i];
                                ab[i] = t;
                                st2[c + i] = fmaf(yi[i], v[i], st2[c + i]);
                            }
                        }
                    } else {  // BWD_VALUE
                        float a0v[16];
                        load16_f32(a.A0 + (long long)n * hp + j, a0v);
                        if (a.S == 1) {
#pragma unroll
                            for (int i = 0; i < 16; i++) {
                                float y0 = tanhf(a0v[i]);
                                ab[i] = (1.f - y0 * y0) * v[i];
                            }
                        } else {
                            float adv[16], ssq[16], ydv[16], cr[16];
                            load16_f32(a.AD + (long long)n * hp + j, adv);
                            load16_f32(a.SSQ + (long long)n * hp + j, ssq);
                            load16_f32(a.YD + (long long)n * hp + j, ydv);
#pragma unroll
                            for (int i = 0; i < 16; i++) cr[i] = 0.f;
                            for (int z = 0; z < a.n_chunks; z++) {
                                float t[16];
                                load16_f32(a.part + ((long long)z * a.N_pad + n) * hp + j, t);
#pragma unroll
                                for (int i = 0; i < 16; i++) cr[i] += t[i];
                            }
#pragma unroll
                            for (int i = 0; i < 16; i++) {
                                float y0 = tanhf(a0v[i]);
                                float s1 = 1.f - y0 * y0;
                                ab[i] = s1 * v[i] - 2.f * y0 * cr[i] -
                                        2.f * s1 * (y0 * adv[i] + (1.f - 3.f * y0 * y0) * ssq[i]) * ydv[i];
                            }
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        if (!live || j + i >= a.n_out) ab[i] = 0.f;
                        gr[i] = rn * ab[i];
                    }
                    if (SPLIT) {
                        float ah[16], al[16], gh[16], gl[16];
#pragma unroll
                        for (int i = 0; i < 16; i++) {
                            __nv_bfloat16 hb;
                            al[i] = bf_round_lo(ab[i], hb);
                            ah[i] = __bfloat162float(hb);
                            gl[i] = bf_round_lo(gr[i], hb);
                            gh[i] = __bfloat162float(hb);
                        }
                        store16_bf16(a.out_hi + ((long long)s * a.N_pad + n) * hp + j, ah);
                        store16_bf16(a.out_lo + ((long long)s * a.N_pad + n) * hp + j, al);
                        store16_bf16(a.out_gr + ((long long)s * a.N_pad + n) * hp + j, gh);
                        store16_bf16(a.out_gr_lo + ((long long)s * a.N_pad + n) * hp + j, gl);
                    } else {
                        store16_bf16(a.out_hi + ((long long)s * a.N_pad + n) * hp + j, ab);
                        store16_bf16(a.out_gr + ((long long)s * a.N_pad + n) * hp + j, gr);
                    }
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (PAIR && rank != 0) tc::mbar_arrive_cluster(tc::mapa_shared(&acc_empty[buf], 0));
                else tc::mbar_arrive(&acc_empty[buf]);
            }
        }
        if (STATE && !abort_flag && !idle) {
#pragma unroll
            for (int c = 0; c < CW; c += 16) {
                const int j = j0 + c0 + c;
                if (j < a.hp_out)
                    store16_f32(a.part + ((long long)vb.z * a.N_pad + n) * hp + j, st2 + c);
            }
        }
        if (MODE == JDOT && !abort_flag) {
            // one partial per (column chunk, feature tile, column half) and point
            const long long slot = ((long long)vb.z * vg.x + vb.x) * 2 + half;
            a.part[slot * a.N_pad + n] = jacc;
        }
    }

    tc::tc_fence_before();
    if (PAIR) tc::cluster_sync();
    else __syncthreads();
    if (abort_flag && threadIdx.x == 0) latch_status(a.status, KFAC_TIMEOUT);
    if (warp == 1) {
        tc::tc_fence_after();
        if (PAIR) tc::tmem_dealloc_pair(tbase, C::TMEM_COLS);
        else tc::tmem_dealloc(tbase, C::TMEM_COLS);
    }
}

template <int MODE, bool SPLIT>
__global__ void __launch_bounds__(NUM_THREADS, 1) tc_engine(const __grid_constant__ Args a) {
    engine_body<MODE, SPLIT>(a, blockIdx, make_uint3(gridDim.x, gridDim.y, gridDim.z));
}

// The forward modes on CTA pairs: grid (2 x feature tiles, point blocks / 2
// rounded up, column chunks).
template <int MODE, bool SPLIT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NUM_THREADS, 1) tc_engine_pair(const __grid_constant__ Args a) {
    engine_body<MODE, SPLIT, true>(a, blockIdx, make_uint3(gridDim.x, gridDim.y, gridDim.z));
}

// Grouped launch (group.cuh): every member's Args, tensor maps included, in a
// table in global memory.  The producer thread acquires the maps for the
// tensor-map proxy before its first TMA through them.
template <int MODE, bool SPLIT>
__global__ void __launch_bounds__(NUM_THREADS, 1) tc_engine_group(const __grid_constant__ GroupTab t) {
    const int m = group_member(t, blockIdx.x);
    const uint3 g = t.grid[m];
    const Args& a = *reinterpret_cast<const Args*>(t.packs + (size_t)m * t.stride);
    if (threadIdx.x == 0) {
        tc::tmap_acquire(&a.a0);
        tc::tmap_acquire(&a.a1);
        tc::tmap_acquire(&a.b0);
        tc::tmap_acquire(&a.b1);
    }
    engine_body<MODE, SPLIT>(a, group_block(blockIdx.x - t.start[m], g), g);
}

// Grouped launch of CTA-pair members: every member's grid.x is even, so its
// first flat block is even and each cluster of two holds blocks 2q and
// 2q + 1 of one member (one feature tile, one pair of point blocks).
template <int MODE, bool SPLIT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NUM_THREADS, 1)
    tc_engine_group_pair(const __grid_constant__ GroupTab t) {
    const int m = group_member(t, blockIdx.x);
    const uint3 g = t.grid[m];
    const Args& a = *reinterpret_cast<const Args*>(t.packs + (size_t)m * t.stride);
    if (threadIdx.x == 0) {
        tc::tmap_acquire(&a.a0);
        tc::tmap_acquire(&a.a1);
        tc::tmap_acquire(&a.b0);
        tc::tmap_acquire(&a.b1);
    }
    engine_body<MODE, SPLIT, true>(a, group_block(blockIdx.x - t.start[m], g), g);
}

}  // namespace tck
