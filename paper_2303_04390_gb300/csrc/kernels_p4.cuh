// FP32 level kernels for 4 padded states (nucleotide models): one thread
// per pattern, covering every rate category.
//
// Arithmetic as in the register kernels of kernels.cuh (Eq. 2 with the
// root's Eq. 3; Eq. 4 with the fused Eq. 8 ratio and Eq. 7 tile sums).  The
// mapping is chosen for S = 4, where a (pattern, category) pair carries too
// little work to pay for per-pair shuffles:
//  - a thread owns one pattern and all R <= RM categories, so the rescale
//    maximum, the sums over categories and the gradient ratio are local;
//  - the thread issues every 16-byte load of its pattern (R vectors per
//    input) before it computes, so each warp keeps 3 x R x 512 bytes in
//    flight;
//  - the block's transition matrices are staged in shared memory by 1-D
//    bulk copies (cp.async.bulk) on an mbarrier, one per child, in the
//    orientations the products read (the matrix kernel writes P', dP' and
//    P per branch), so that P v, dP v and P' a all run on the packed FP32
//    FMA (__ffma2_rn, two lanes per instruction) from 16-byte broadcast
//    reads;
//  - partials are tile-blocked ([slot][tile][r][32][4], phylo_internal.h),
//    so each warp's access of one category is 512 contiguous bytes;
//  - a tile's (warp's) gradient sums are FP32 pairs kept exact with
//    error-free transformations (converted to FP64 by the final reduction).
// The U form: the post-order step of a (non-cherry, non-root) node k stores
// U_k = P_k p_k, the factor k contributes to its parent in Eq. 2, instead of
// p_k, so its parent reads U_k where it read p_k (the same bytes) and skips
// that product; in the pre-order step such a child's Eq. 8 numerator is
// gamma_r (a' Q) U (q' Q p with q = P' a, P = exp(gamma_r t Q) commuting
// with Q): one product where P p and dP p were two.  Cherries, tips with
// partial vectors and compact tips keep the p form (their U, dP p or
// columns are formed from the tip data in the step that needs them).
#pragma once

namespace phylo {

constexpr int kP4Threads = 64;  // patterns per block: two tiles

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// out = M v for 4x4 M given by the rows of M' (t-th row = column t of M).
__device__ __forceinline__ void mv4t(const float4* __restrict__ MT, float4 v,
                                     float2& lo, float2& hi) {
  const float4 c0 = MT[0], c1 = MT[1], c2 = MT[2], c3 = MT[3];
  lo = __fmul2_rn(lo2(c0), make_float2(v.x, v.x));
  hi = __fmul2_rn(hi2(c0), make_float2(v.x, v.x));
  lo = __ffma2_rn(lo2(c1), make_float2(v.y, v.y), lo);
  hi = __ffma2_rn(hi2(c1), make_float2(v.y, v.y), hi);
  lo = __ffma2_rn(lo2(c2), make_float2(v.z, v.z), lo);
  hi = __ffma2_rn(hi2(c2), make_float2(v.z, v.z), hi);
  lo = __ffma2_rn(lo2(c3), make_float2(v.w, v.w), lo);
  hi = __ffma2_rn(hi2(c3), make_float2(v.w, v.w), hi);
}

// out = M' a for 4x4 M given by its rows.
__device__ __forceinline__ void mtv4r(const float4* __restrict__ M, float2 alo,
                                      float2 ahi, float2& lo, float2& hi) {
  const float4 r0 = M[0], r1 = M[1], r2 = M[2], r3 = M[3];
  lo = __fmul2_rn(lo2(r0), make_float2(alo.x, alo.x));
  hi = __fmul2_rn(hi2(r0), make_float2(alo.x, alo.x));
  lo = __ffma2_rn(lo2(r1), make_float2(alo.y, alo.y), lo);
  hi = __ffma2_rn(hi2(r1), make_float2(alo.y, alo.y), hi);
  lo = __ffma2_rn(lo2(r2), make_float2(ahi.x, ahi.x), lo);
  hi = __ffma2_rn(hi2(r2), make_float2(ahi.x, ahi.x), hi);
  lo = __ffma2_rn(lo2(r3), make_float2(ahi.y, ahi.y), lo);
  hi = __ffma2_rn(hi2(r3), make_float2(ahi.y, ahi.y), hi);
}

__device__ __forceinline__ float dot22(float2 alo, float2 ahi, float2 blo,
                                       float2 bhi) {
  float2 x = __fmul2_rn(alo, blo);
  x = __ffma2_rn(ahi, bhi, x);
  return x.x + x.y;
}

__device__ __forceinline__ float max4(float2 lo, float2 hi) {
  return fmaxf(fmaxf(fabsf(lo.x), fabsf(lo.y)), fmaxf(fabsf(hi.x), fabsf(hi.y)));
}

// Shared layout of one block.  m[x] holds child x's branch block as the
// matrix kernel wrote it: P' of every category (R x 16 floats) and, for the
// pre-order step, dP' and P after it (float4 offsets 0, 4R and 8R).  g holds
// P' of the tip branches below a cherry child (i: 0, 1; j: 2, 3).  n holds
// the node's own P' (post-order: U_k = P_k p_k) or Q (pre-order, one
// matrix: the Eq. 8 numerator of a child whose U is stored).
template <int RM, bool PRE, bool CH>
struct P4Mats {
  float4 m[2][(PRE ? kP4MatKinds : 1) * RM * 4];
  float4 g[CH ? 4 : 1][RM * 4];
  float4 n[PRE ? 4 : RM * 4];
};

// Power-of-two rescale of a vector whose largest magnitude is mx (finite,
// > 0): returns e with mx = f 2^e, f in [0.5, 1) (as frexp), and sets
// s = 2^-e.  Normal mx reads the exponent field; subnormal or huge mx takes
// frexpf/ldexpf.
__device__ __forceinline__ int p4_rescale(float mx, float& s) {
  const int b = (__float_as_int(mx) >> 23) & 0xff;
  if (b >= 1 && b <= 252) {
    s = __int_as_float((253 - b) << 23);
    return b - 126;
  }
  int e;
  (void)frexpf(mx, &e);
  s = ldexpf(1.f, -e);
  return e;
}

// Cherry fusion.  A cherry is a non-root internal node whose two children
// are tips with compact states.  It gets no post-order launch and stores no
// partials: wherever its partials are needed (its parent's post- and
// pre-order steps) they are formed as p_x = (P_xa e_ya) o (P_xb e_yb) from
// the two tip states (no rescale is needed: both factors are transition
// probabilities).  This removes the write of p_x and its two read-backs.
// The cherry keeps its own pre-order step.
__device__ __forceinline__ float4 p4_col(const float4* T, int y, int S) {
  if (y < S) return T[y];
  return make_float4(1.f, S > 1 ? 1.f : 0.f, S > 2 ? 1.f : 0.f, S > 3 ? 1.f : 0.f);
}

// The child's 4 states for category r: u = M v (and w = dM v), a compact
// state selecting a column (gap: all ones, w = 0).
template <bool WITH_D>
__device__ __forceinline__ void p4_child(int y, int S, float4 v,
                                         const float4* MT, const float4* DT,
                                         float2& ulo, float2& uhi, float2& wlo,
                                         float2& whi) {
  if (y >= 0) {
    if (y < S) {
      const float4 col = MT[y];
      ulo = lo2(col); uhi = hi2(col);
      if (WITH_D) { const float4 dc = DT[y]; wlo = lo2(dc); whi = hi2(dc); }
    } else {
      ulo = make_float2(1.f, S > 1 ? 1.f : 0.f);
      uhi = make_float2(S > 2 ? 1.f : 0.f, S > 3 ? 1.f : 0.f);
      if (WITH_D) { wlo = make_float2(0.f, 0.f); whi = wlo; }
    }
    return;
  }
  mv4t(MT, v, ulo, uhi);
  if (WITH_D) mv4t(DT, v, wlo, whi);
}

// The pre-order kernel is latency-bound at these occupancies: in the p form
// asking for 12 resident blocks per SM (at most 85 registers a thread)
// measured 4% faster than the unbounded register allocation; in the U form
// that bound spills and 11 blocks (at most 88 registers) measured best
// (hky-1024 pre-order 0.434 ms; 12 blocks 0.444, 10 blocks 0.467).  The
// post-order kernel is left unbounded.
#ifndef PHYLO_P4_PRE_BLOCKS
#define PHYLO_P4_PRE_BLOCKS 11
#endif
constexpr int kP4PreMinBlocks = PHYLO_P4_PRE_BLOCKS;

// RM: categories unrolled (R <= RM); EX: R == RM, so that no per-category
// test is left at run time.
template <int RM, bool EX, bool PRE, bool CH>
__global__ void __launch_bounds__(kP4Threads, PRE ? kP4PreMinBlocks : 0)
    level_p4_kernel(LevelArgs<float> a) {
  __shared__ P4Mats<RM, PRE, CH> sm;
  __shared__ uint64_t bar;
  const int tid = threadIdx.x, lane = tid & 31;
  const int R = EX ? RM : a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x, bi = d.y, bj = d.z;
  const bool ci = d.w & kDescFlagCompact0, cj = d.w & kDescFlagCompact1;
  const bool hi_ = CH && (d.w & kDescFlagCherry0), hj_ = CH && (d.w & kDescFlagCherry1);
  const int2 gi2 = hi_ ? a.children[bi] : make_int2(0, 0);  // tips below a cherry
  const int2 gj2 = hj_ ? a.children[bj] : make_int2(0, 0);
  const int c = blockIdx.x * kP4Threads + tid;
  const int tile = c >> 5;  // this warp's tile
  const bool valid = c < C;
  const uint32_t mbytes = (uint32_t)R * 64;  // one matrix of every category
  const uint32_t cbytes = (PRE ? kP4MatKinds : 1) * mbytes;  // a child's block
  const size_t bstride = (size_t)kP4MatKinds * R * 16;      // floats per branch
  if (tid == 0) mbar_init_fenced(&bar, 1);
  __syncthreads();
  // The descriptor, the tree and the tip states are written by the host and
  // read before the wait; so are the matrices when the launch before this
  // one is not the matrix kernel.
  auto issue_copies = [&] {
    if (tid != 0) return;
    const int n_ch = (int)hi_ + (int)hj_;
    // the node's own P' (post-order, not at the root) or Q (pre-order)
    const uint32_t nbytes = PRE ? 64u : (k != a.root ? mbytes : 0u);
    mbar_expect_tx(&bar, 2 * cbytes + 2 * n_ch * mbytes + nbytes);
    bulk_g2s(sm.m[0], a.P + (size_t)bi * bstride, cbytes, &bar);
    bulk_g2s(sm.m[1], a.P + (size_t)bj * bstride, cbytes, &bar);
    if (nbytes) bulk_g2s(sm.n, PRE ? a.qmat : a.P + (size_t)k * bstride, nbytes, &bar);
    if constexpr (CH) {
      for (int x = 0; x < 2; ++x) {
        if (!(x == 0 ? hi_ : hj_)) continue;
        const int2 g = x == 0 ? gi2 : gj2;
        bulk_g2s(sm.g[2 * x], a.P + (size_t)g.x * bstride, mbytes, &bar);
        bulk_g2s(sm.g[2 * x + 1], a.P + (size_t)g.y * bstride, mbytes, &bar);
      }
    }
  };
  if (a.mats_ready) issue_copies();
  // ---- every global load of this pattern, issued before any use ----------
  float4 vi[RM], vj[RM], q[RM];
  int yi = -1, yj = -1, ei = 0, ej = 0;
  int ya[2] = {0, 0}, yb[2] = {0, 0};  // tip states below cherry children
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) {
    if (ci) yi = a.tip_states[(size_t)bi * a.state_stride + c];
    if (cj) yj = a.tip_states[(size_t)bj * a.state_stride + c];
    if (hi_) {
      ya[0] = a.tip_states[(size_t)gi2.x * a.state_stride + c];
      yb[0] = a.tip_states[(size_t)gi2.y * a.state_stride + c];
    }
    if (hj_) {
      ya[1] = a.tip_states[(size_t)gj2.x * a.state_stride + c];
      yb[1] = a.tip_states[(size_t)gj2.y * a.state_stride + c];
    }
  }
  pdl_wait_and_release();
  if (!a.mats_ready) issue_copies();
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    const bool on = valid && r < R;
    vi[r] = zero4; vj[r] = zero4; q[r] = zero4;
    if (on && !ci && !hi_)
      vi[r] = bi < a.n_tips ? __ldg(reinterpret_cast<const float4*>(a.tip_partials) + (size_t)bi * C + c)
                            : __ldg(reinterpret_cast<const float4*>(a.post) +
                                    p4_index(bi - a.n_tips, c, r, R, a.n_tiles));
    if (on && !cj && !hj_)
      vj[r] = bj < a.n_tips ? __ldg(reinterpret_cast<const float4*>(a.tip_partials) + (size_t)bj * C + c)
                            : __ldg(reinterpret_cast<const float4*>(a.post) +
                                    p4_index(bj - a.n_tips, c, r, R, a.n_tiles));
    if (PRE && on && k != a.root)
      q[r] = __ldg(reinterpret_cast<const float4*>(a.pre) +
                   p4_index(k - a.n_tips, c, r, R, a.n_tiles));
  }
  if (PRE && k == a.root) {  // Eq. 4 at the root: q = pi
    const float4 pr = make_float4(a.root_pit[0], S > 1 ? a.root_pit[1] : 0.f,
                                  S > 2 ? a.root_pit[2] : 0.f, S > 3 ? a.root_pit[3] : 0.f);
#pragma unroll
    for (int r = 0; r < RM; ++r) q[r] = pr;
  }
  if (!PRE && valid) {  // a cherry's exponent is 0 (its partials are not rescaled)
    if (bi >= a.n_tips && !hi_) ei = a.escale[(size_t)(bi - a.n_tips) * a.escale_stride + c];
    if (bj >= a.n_tips && !hj_) ej = a.escale[(size_t)(bj - a.n_tips) * a.escale_stride + c];
  }
  // ---- matrices: wait for the bulk copies ---------------------------------
  if (!__syncthreads_and(mbar_wait(&bar, 0))) {
    if (tid == 0) atomicOr(a.err, ERR_TIMEOUT);
    return;
  }
  // child x's P', dP' and P of category r
  const float4* PTi = sm.m[0];
  const float4* PTj = sm.m[1];
  const float4* DTi = sm.m[0] + (PRE ? 4 * R : 0);  // (post-order: unused)
  const float4* DTj = sm.m[1] + (PRE ? 4 * R : 0);
  const float4* Pi = sm.m[0] + (PRE ? 8 * R : 0);
  const float4* Pj = sm.m[1] + (PRE ? 8 * R : 0);
  if constexpr (CH) {
    // a cherry child's partials from its two tip states
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      if (!(valid && r < R)) continue;
      if (hi_) {
        const float4 u = p4_col(sm.g[0] + r * 4, ya[0], S), w = p4_col(sm.g[1] + r * 4, yb[0], S);
        vi[r] = make_float4(u.x * w.x, u.y * w.y, u.z * w.z, u.w * w.w);
      }
      if (hj_) {
        const float4 u = p4_col(sm.g[2] + r * 4, ya[1], S), w = p4_col(sm.g[3] + r * 4, yb[1], S);
        vj[r] = make_float4(u.x * w.x, u.y * w.y, u.z * w.z, u.w * w.w);
      }
    }
  }
  // children whose U = P p is stored (non-cherry internal nodes)
  const bool su_i = bi >= a.n_tips && !hi_, su_j = bj >= a.n_tips && !hj_;
  if (!PRE) {
    // ---- Eq. 2: p_k = U_i o U_j for every category -------------------------
    float2 plo[RM], phi[RM];
    float m = 0.f;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      plo[r] = make_float2(0.f, 0.f); phi[r] = plo[r];
      if (r < R) {
        float2 ilo, ihi, jlo, jhi, d0, d1;
        if (su_i) { ilo = lo2(vi[r]); ihi = hi2(vi[r]); }
        else p4_child<false>(yi, S, vi[r], PTi + r * 4, nullptr, ilo, ihi, d0, d1);
        if (su_j) { jlo = lo2(vj[r]); jhi = hi2(vj[r]); }
        else p4_child<false>(yj, S, vj[r], PTj + r * 4, nullptr, jlo, jhi, d0, d1);
        plo[r] = __fmul2_rn(ilo, jlo);
        phi[r] = __fmul2_rn(ihi, jhi);
        m = fmaxf(m, max4(plo[r], phi[r]));
      }
    }
    int e = 0;
    float f = 1.f;
    if (valid) {
      if (!(m > 0.f) || !isfinite(m)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      else e = p4_rescale(m, f);
    }
    e += ei + ej;
    if (k != a.root) {
      if (valid) {  // U_k = P_k p_k, stored with p_k's exponent
        float4* out = reinterpret_cast<float4*>(a.post) + p4_index(k - a.n_tips, c, 0, R, a.n_tiles);
#pragma unroll
        for (int r = 0; r < RM; ++r)
          if (r < R) {
            const float2 lo = __fmul2_rn(plo[r], make_float2(f, f));
            const float2 hi = __fmul2_rn(phi[r], make_float2(f, f));
            float2 ulo, uhi;
            mv4t(sm.n + r * 4, make_float4(lo.x, lo.y, hi.x, hi.y), ulo, uhi);
            out[32 * r] = make_float4(ulo.x, ulo.y, uhi.x, uhi.y);
          }
        a.escale[(size_t)(k - a.n_tips) * a.escale_stride + c] = e;
      }
      return;
    }
    // Eq. 3 at the root: L_c = sum_r w_r pi' p_root,r,c, exponents restored
    double term = 0.0;
    if (valid) {
      const float2 pl = make_float2(a.root_pit[0], S > 1 ? a.root_pit[1] : 0.f);
      const float2 ph = make_float2(S > 2 ? a.root_pit[2] : 0.f, S > 3 ? a.root_pit[3] : 0.f);
      float L = 0.f;
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < R) L = fmaf(a.cat_wt[r], dot22(pl, ph, plo[r], phi[r]) * f, L);
      if (!(L > 0.f) || !isfinite(L)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      term = (double)a.pattern_wt[c] * (log((double)L) + (double)e * 0.69314718055994530942);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(kFull, term, o);
    if (lane == 0 && tile < a.n_tiles) a.lpart[tile] = term;
    return;
  }
  // ---- Eq. 4 and Eq. 8: children's pre-order partials and the ratio ------
  const bool int_i = bi >= a.n_tips, int_j = bj >= a.n_tips;
  float2 qilo[RM], qihi[RM], qjlo[RM], qjhi[RM];
  float Ni = 0.f, Nj = 0.f, Dn = 0.f, mi = 0.f, mj = 0.f;
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    qilo[r] = make_float2(0.f, 0.f); qihi[r] = qilo[r]; qjlo[r] = qilo[r]; qjhi[r] = qilo[r];
    if (r < R) {
      const float2 ql = lo2(q[r]), qh = hi2(q[r]);
      float2 uilo, uihi, wilo, wihi, ujlo, ujhi, wjlo, wjhi;
      // a stored U needs no product here; the others give U and dP p (or columns)
      if (su_i) { uilo = lo2(vi[r]); uihi = hi2(vi[r]); }
      else p4_child<true>(yi, S, vi[r], PTi + r * 4, DTi + r * 4, uilo, uihi, wilo, wihi);
      if (su_j) { ujlo = lo2(vj[r]); ujhi = hi2(vj[r]); }
      else p4_child<true>(yj, S, vj[r], PTj + r * 4, DTj + r * 4, ujlo, ujhi, wjlo, wjhi);
      const float2 ailo = __fmul2_rn(ql, ujlo), aihi = __fmul2_rn(qh, ujhi);  // a_i
      const float2 ajlo = __fmul2_rn(ql, uilo), ajhi = __fmul2_rn(qh, uihi);  // a_j
      const float w = a.cat_wt[r];
      float ni, nj;
      if (su_i || su_j) {
        const float gam = (float)a.rates[r];
        float2 lo, hi;
        if (su_i) {  // gamma_r (a_i' Q) U_i
          mtv4r(sm.n, ailo, aihi, lo, hi);
          ni = gam * dot22(lo, hi, uilo, uihi);
        }
        if (su_j) {
          mtv4r(sm.n, ajlo, ajhi, lo, hi);
          nj = gam * dot22(lo, hi, ujlo, ujhi);
        }
      }
      if (!su_i) ni = dot22(ailo, aihi, wilo, wihi);
      if (!su_j) nj = dot22(ajlo, ajhi, wjlo, wjhi);
      Ni = fmaf(w, ni, Ni);
      Nj = fmaf(w, nj, Nj);
      Dn = fmaf(w, dot22(ailo, aihi, uilo, uihi), Dn);
      if (int_i) {
        mtv4r(Pi + r * 4, ailo, aihi, qilo[r], qihi[r]);
        mi = fmaxf(mi, max4(qilo[r], qihi[r]));
      }
      if (int_j) {
        mtv4r(Pj + r * 4, ajlo, ajhi, qjlo[r], qjhi[r]);
        mj = fmaxf(mj, max4(qjlo[r], qjhi[r]));
      }
    }
  }
  F2 gi = {0.f, 0.f}, gj = {0.f, 0.f};
  if (valid) {
    if (!(Dn > 0.f) || !isfinite(Dn)) {
      atomicOr(a.err, ERR_BAD_RATIO);
    } else {
      const float W = a.pattern_wt[c], rd = __fdividef(1.f, Dn);  // Dn << 2^126
      gi = Acc<float>::prod(W, Ni * rd);
      gj = Acc<float>::prod(W, Nj * rd);
    }
    if (int_i) {
      float f = 1.f;
      if (!(mi > 0.f) || !isfinite(mi)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      else (void)p4_rescale(mi, f);
      float4* out = reinterpret_cast<float4*>(a.pre) + p4_index(bi - a.n_tips, c, 0, R, a.n_tiles);
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < R) {
          const float2 lo = __fmul2_rn(qilo[r], make_float2(f, f));
          const float2 hi = __fmul2_rn(qihi[r], make_float2(f, f));
          out[32 * r] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
    }
    if (int_j) {
      float f = 1.f;
      if (!(mj > 0.f) || !isfinite(mj)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      else (void)p4_rescale(mj, f);
      float4* out = reinterpret_cast<float4*>(a.pre) + p4_index(bj - a.n_tips, c, 0, R, a.n_tiles);
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < R) {
          const float2 lo = __fmul2_rn(qjlo[r], make_float2(f, f));
          const float2 hi = __fmul2_rn(qjhi[r], make_float2(f, f));
          out[32 * r] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
    }
  }
  // Both children's tile sums in one butterfly: after the first exchange
  // lanes 0-15 carry child i's pairs and lanes 16-31 child j's, so each
  // later level moves and adds one pair instead of two.
  {
    const bool upper = lane >= 16;
    F2 mine = upper ? gj : gi;
    const F2 other = upper ? gi : gj;
    mine = f2_add(mine, F2{__shfl_xor_sync(kFull, other.hi, 16),
                           __shfl_xor_sync(kFull, other.lo, 16)});
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mine = f2_add(mine, Acc<float>::shfl_down(mine, o));
    // the pair as stored (the reduction converts to FP64: no FP64 here)
    float2* gp = reinterpret_cast<float2*>(a.gpart);
    if (tile < a.n_tiles && (lane == 0 || lane == 16))
      gp[(size_t)(lane == 0 ? bi : bj) * a.n_tiles + tile] = make_float2(mine.hi, mine.lo);
  }
}

template <int RM, bool EX>
cudaError_t launch_p4_ex(const LevelArgs<float>& a, bool post, cudaStream_t st) {
  dim3 grid((a.n_tiles + 1) / 2, a.n_level);
  if (a.level_cherry) {
    if (post) return launch_pdl(level_p4_kernel<RM, EX, false, true>, grid, kP4Threads, 0, st, a);
    return launch_pdl(level_p4_kernel<RM, EX, true, true>, grid, kP4Threads, 0, st, a);
  }
  if (post) return launch_pdl(level_p4_kernel<RM, EX, false, false>, grid, kP4Threads, 0, st, a);
  return launch_pdl(level_p4_kernel<RM, EX, true, false>, grid, kP4Threads, 0, st, a);
}

template <int RM>
cudaError_t launch_p4(const LevelArgs<float>& a, bool post, cudaStream_t st) {
  if (a.n_cat == RM) return launch_p4_ex<RM, true>(a, post, st);
  if constexpr (RM > 2) return launch_p4_ex<RM, false>(a, post, st);
  return cudaErrorInvalidValue;
}

// RP (next power of two >= R) selects the unrolled category count.
inline cudaError_t launch_p4_rp(const LevelArgs<float>& a, int RP, bool post,
                                cudaStream_t st) {
  switch (RP) {
    case 1: return launch_p4<1>(a, post, st);
    case 2: return launch_p4<2>(a, post, st);
    case 4: return launch_p4<4>(a, post, st);
    case 8: return launch_p4<8>(a, post, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace phylo
