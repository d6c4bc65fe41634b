// Time-axis kernels of the ParaDiag-II preconditioner (steps (a) and (c) of
// eq. 1.3 / eq. 2.12):
//   K1  r -> Gamma_alpha r -> FFT along t (half spectrum of a real signal),
//       optionally fused with the all-at-once residual r = b - A u (eq. 5.1);
//   K3  inverse FFT along t -> Gamma_alpha^{-1}/Nt -> write z or update u += z.
// One block owns a tile of TX consecutive spatial columns over all Nt time
// levels.  Two real columns are packed into one complex column (even x -> real,
// odd x -> imaginary part), transformed by a shared-memory Stockham FFT
// (radix 4 with one radix-2 pass when log2 Nt is odd), and separated with
// A_k = (Z_k + conj Z_{N-k})/2, B_k = (Z_k - conj Z_{N-k})/(2i).
// The transform convention is the forward DFT with exp(-2 pi i k n / Nt); the
// eigenvalues used in step (b) follow the same convention (see pd_api.cu).
#include <type_traits>

#include "pd_internal.h"

namespace {

constexpr int TT = 256;  // threads per block

template <int BYTES>
PD_D void cp_async(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
PD_D void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// ---- thread-block clusters: rank, barrier, distributed shared memory
PD_D int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}
// every thread of every block of the cluster; orders the shared-memory
// writes before it (local and remote) before the reads after it
PD_D void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of the same shared-memory offset in block `rank`
PD_D uint32_t dsm_map(const void* p, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
PD_D float2 dsm_ld(uint32_t a, float2) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
}
PD_D double2 dsm_ld(uint32_t a, double2) {
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
  return v;
}
PD_D void dsm_st(uint32_t a, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
PD_D void dsm_st(uint32_t a, double2 v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}

template <typename C, bool INV>
PD_D C twid(const C* tw, int idx) {
  C w = tw[idx];
  if (INV) w.y = -w.y;
  return w;
}

// v * exp(-+2 pi i e / 16) for a compile-time e (INV: the + sign)
template <typename C, bool INV, int E>
PD_D C w16(C v) {
  using R = decltype(v.x);
  constexpr int e = E & 15;
  if constexpr (e == 0) {
    return v;
  } else if constexpr (e == 4) {
    return INV ? cmul_pi(v) : cmul_mi(v);
  } else if constexpr (e == 8) {
    return mk(-v.x, -v.y);
  } else if constexpr (e == 12) {
    return INV ? cmul_mi(v) : cmul_pi(v);
  } else {
    // cos and sin of 2 pi e / 16 from the values at pi/8, pi/4 and 3 pi/8
    constexpr double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173;
    constexpr double H = 0.70710678118654752440;
    constexpr int q = e & 3;  // position inside the quadrant
    constexpr double cb = q == 1 ? C1 : q == 2 ? H : S1;
    constexpr double sb = q == 1 ? S1 : q == 2 ? H : C1;
    // rotate the first-quadrant angle by the quadrant index e / 4
    constexpr int quad = e >> 2;
    constexpr double c0 = quad == 0 ? cb : quad == 1 ? -sb : quad == 2 ? -cb : sb;
    constexpr double s0 = quad == 0 ? sb : quad == 1 ? cb : quad == 2 ? -sb : -cb;
    const R c = (R)c0, s = INV ? (R)s0 : (R)-s0;
    return mk(v.x * c - v.y * s, v.x * s + v.y * c);
  }
}

// in-register DFT of size R (2, 4, 8, 16) with the exp(-+2 pi i / R) root
template <typename C, bool INV, int R>
PD_D void dft_r(C* v) {
  if constexpr (R == 2) {
    C a = cadd(v[0], v[1]), b = csub(v[0], v[1]);
    v[0] = a; v[1] = b;
  } else if constexpr (R == 4) {
    C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    C s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
    C jd13 = INV ? cmul_pi(d13) : cmul_mi(d13);  // (-+i)(x1 - x3)
    v[0] = cadd(s02, s13);
    v[1] = cadd(d02, jd13);
    v[2] = csub(s02, s13);
    v[3] = csub(d02, jd13);
  } else if constexpr (R == 8) {
    // n = 2 n1 + n2, k = k1 + 4 k2: DFT-4 over n1, twiddle W8^(n2 k1), DFT-2 over n2
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft_r<C, INV, 4>(e);
    dft_r<C, INV, 4>(o);
    o[1] = w16<C, INV, 2>(o[1]);
    o[2] = w16<C, INV, 4>(o[2]);
    o[3] = w16<C, INV, 6>(o[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  } else {
    // n = 4 n1 + n2, k = k1 + 4 k2: DFT-4 over n1, twiddle W16^(n2 k1), DFT-4 over n2
    C y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      y[n2][0] = v[n2]; y[n2][1] = v[4 + n2]; y[n2][2] = v[8 + n2]; y[n2][3] = v[12 + n2];
      dft_r<C, INV, 4>(y[n2]);
    }
    y[1][1] = w16<C, INV, 1>(y[1][1]);
    y[1][2] = w16<C, INV, 2>(y[1][2]);
    y[1][3] = w16<C, INV, 3>(y[1][3]);
    y[2][1] = w16<C, INV, 2>(y[2][1]);
    y[2][2] = w16<C, INV, 4>(y[2][2]);
    y[2][3] = w16<C, INV, 6>(y[2][3]);
    y[3][1] = w16<C, INV, 3>(y[3][1]);
    y[3][2] = w16<C, INV, 6>(y[3][2]);
    y[3][3] = w16<C, INV, 9>(y[3][3]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      C z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      dft_r<C, INV, 4>(z);
      v[k1] = z[0]; v[k1 + 4] = z[1]; v[k1 + 8] = z[2]; v[k1 + 12] = z[3];
    }
  }
}

// One Stockham pass of radix R = 2^LR over TXc interleaved columns stored
// [N][TXc].  Butterfly b = (j << lgTXc) + c (column c, index j < N/R) reads
// rows j + r N/R, applies the twiddles w_N^(q r N/(R Ns)) with q = j mod Ns,
// and writes rows (j - q) R + q + k Ns; with every size a power of two all the
// index arithmetic is shifts and masks.  Every butterfly is read into
// registers before the barrier and written after it, so the pass runs in place.
template <typename C, bool INV, int LR, int BPT, bool FIRST = false>
PD_D void fft_pass(C* sm, int lgN, int lgTXc, int lgNs, const C* tw) {
  constexpr int R = 1 << LR;
  const int lgNB = lgN - LR + lgTXc;        // butterflies: (N / R) TXc
  const int nb = 1 << lgNB;
  const int lgStep = lgN - LR - lgNs;
  const int lgOut = lgNs + lgTXc;
  const int lomask = (1 << lgOut) - 1;
  const int qmask = (1 << lgNs) - 1;
  C v[BPT][R];
  int dst[BPT];
#pragma unroll
  for (int t = 0; t < BPT; ++t) {
    const int b = threadIdx.x + t * TT;
    dst[t] = -1;
    if (b < nb) {
      const int tq = ((b >> lgTXc) & qmask) << lgStep;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = sm[b + (r << lgNB)];
        if (!FIRST && r > 0) x = cmul(x, twid<C, INV>(tw, tq * r));
        v[t][r] = x;
      }
      dft_r<C, INV, R>(v[t]);
      const int lo = b & lomask;
      dst[t] = ((b - lo) << LR) + lo;
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < BPT; ++t) {
    if (dst[t] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) sm[dst[t] + (r << lgOut)] = v[t][r];
    }
  }
  __syncthreads();
}

// Full complex FFT of length N = 2^logN on TXc columns: one pass of radix
// 2, 4 or 8 for logN mod 4, then radix-16 passes; EPT is the maximum number of
// complex elements per thread (N TXc <= EPT TT).
template <typename C, bool INV, int EPT>
PD_D void fft_tile(C* sm, int N, int logN, int lgTXc, const C* tw) {
  (void)N;
  constexpr int B16 = EPT / 16 > 0 ? EPT / 16 : 1;
  constexpr int B8 = EPT / 8 > 0 ? EPT / 8 : 1;
  constexpr int B4 = EPT / 4 > 0 ? EPT / 4 : 1;
  constexpr int B2 = EPT / 2 > 0 ? EPT / 2 : 1;
  // the first pass (sub-transform length 1) has unit twiddles
  const int rem = logN & 3;
  if (rem == 1) fft_pass<C, INV, 1, B2, true>(sm, logN, lgTXc, 0, tw);
  else if (rem == 2) fft_pass<C, INV, 2, B4, true>(sm, logN, lgTXc, 0, tw);
  else if (rem == 3) fft_pass<C, INV, 3, B8, true>(sm, logN, lgTXc, 0, tw);
  else if (logN >= 4) fft_pass<C, INV, 4, B16, true>(sm, logN, lgTXc, 0, tw);
  int lgNs = rem != 0 ? rem : (logN >= 4 ? 4 : 0);
  for (; lgNs < logN; lgNs += 4) fft_pass<C, INV, 4, B16>(sm, logN, lgTXc, lgNs, tw);
}

// Length-N DFT of TXc columns by Bluestein's algorithm: a_n = z_n w_n (zero
// padded to M), A = FFT_M(a), A *= bhat, c = inverse FFT_M(A) (the 1/M is in
// bhat), Z_k = w_k c_k.  CONJ computes conj(DFT(conj(z))), the unnormalised
// inverse DFT.  Rows N..M-1 of the tile are scratch.
template <typename C, bool CONJ, int EPT>
PD_D void bluestein_tile(C* sm, int N, const TimeXf& xf, int lgTXc, const C* twM) {
  const C* chirp = reinterpret_cast<const C*>(xf.chirp);
  const C* bhat = reinterpret_cast<const C*>(xf.bhat);
  const int tot = xf.M << lgTXc;
  for (int e = threadIdx.x; e < tot; e += TT) {
    const int n = e >> lgTXc;
    C v = czero<C>();
    if (n < N) {
      v = sm[e];
      if (CONJ) v = cconj(v);
      v = cmul(v, chirp[n]);
    }
    sm[e] = v;
  }
  __syncthreads();
  fft_tile<C, false, EPT>(sm, xf.M, xf.logM, lgTXc, twM);
  for (int e = threadIdx.x; e < tot; e += TT) sm[e] = cmul(sm[e], bhat[e >> lgTXc]);
  __syncthreads();
  fft_tile<C, true, EPT>(sm, xf.M, xf.logM, lgTXc, twM);
  for (int e = threadIdx.x; e < (N << lgTXc); e += TT) {
    C v = cmul(sm[e], chirp[e >> lgTXc]);
    if (CONJ) v = cconj(v);
    sm[e] = v;
  }
  __syncthreads();
}

// One radix-CR step of a length-N transform split over the CR blocks of a
// thread-block cluster; block c holds rows [c L, c L + L) (L = N / CR) of the
// tile [L][TXc] in its shared memory.  With n = t + L c and k = CR k' + j:
//   forward  X_{CR k' + j} = sum_t W_L^{t k'} (W_N^{t j} sum_c x_{t + L c} W_CR^{c j}),
//   inverse  x_{t + L c}   = sum_j W_CR^{-c j} W_N^{-t j} (sum_k' X_{CR k' + j} W_L^{-t k'}),
// W_m = exp(-2 pi i / m).  Forward: this step forms the bracket and writes
// its j-th value of row t into block j; every block then transforms its L
// rows (output k' in natural order).  Inverse: every block first
// inverse-transforms its L rows (k' -> t); this step applies the twiddle and
// the length-CR sum and writes x_{t + L c} into block c.  Block b takes the
// rows t in [b L/CR, (b+1) L/CR) of every block, and the thread that reads
// element (t, column) of each block is the one that writes it, so the step
// runs in place.  The caller brackets it with cluster barriers.  tw is the
// length-N table W_N^m, m < N.
template <typename C, bool INV, int CR>
PD_D void cluster_radix(C* sm, int L, int lgTXc, const C* __restrict__ tw, int rank) {
  const int per = (L / CR) << lgTXc;
  const int e0 = rank * per;
  uint32_t rb[CR];
#pragma unroll
  for (int c = 0; c < CR; ++c) rb[c] = dsm_map(sm, c);
  for (int e = threadIdx.x; e < per; e += TT) {
    const int idx = e0 + e;
    const int t = idx >> lgTXc;
    const uint32_t off = (uint32_t)idx * (uint32_t)sizeof(C);
    C v[CR];
#pragma unroll
    for (int c = 0; c < CR; ++c) v[c] = dsm_ld(rb[c] + off, C{});
    if (!INV) {
      dft_r<C, false, CR>(v);
#pragma unroll
      for (int j = 1; j < CR; ++j) v[j] = cmul(v[j], tw[t * j]);
    } else {
#pragma unroll
      for (int j = 1; j < CR; ++j) v[j] = cmul(v[j], twid<C, true>(tw, t * j));
      dft_r<C, true, CR>(v);
    }
#pragma unroll
    for (int c = 0; c < CR; ++c) dsm_st(rb[c] + off, v[c]);
  }
}

// ---------------------------------------------------------------------------
// Spatial stencil of one time row at this thread's column, x-neighbours from
// the lanes of the same TX-wide segment (warp shuffles), y-neighbours and
// segment edges from global memory.
// ---------------------------------------------------------------------------
struct ColGeom {
  int s;          // spatial index (may be >= S for padding columns)
  bool valid;
  int left;       // 0: zero, 1: from lane - 1, 2: load s_left
  int right;
  int s_left, s_right;
  bool down, up;  // y neighbours present (2D)
};

PD_D ColGeom col_geom(const Stencil& st, int s, int lane_in_seg, int TX) {
  ColGeom g;
  g.s = s;
  g.valid = s < st.S;
  g.left = g.right = 0;
  g.s_left = g.s_right = 0;
  g.down = g.up = false;
  if (!g.valid) return g;
  const int xg = s % st.nx;
  const int y = s / st.nx;
  if (xg > 0) {
    g.left = lane_in_seg > 0 ? 1 : 2;
    g.s_left = s - 1;
  } else if (st.bcx == PD_PERIODIC && st.nx > 1) {
    g.left = 2;
    g.s_left = s + st.nx - 1;
  }
  if (xg < st.nx - 1) {
    g.right = lane_in_seg < TX - 1 ? 1 : 2;
    g.s_right = s + 1;
  } else if (st.bcx == PD_PERIODIC && st.nx > 1) {
    g.right = 2;
    g.s_right = s - (st.nx - 1);
  }
  if (st.dim == 2) {
    g.down = y > 0;
    g.up = y < st.ny - 1;
  }
  return g;
}

struct Acc {  // compensated sum: value = s + e
  float s, e;
};
PD_D void acc_add(Acc& A, float h, float l) {
  const float t = __fadd_rn(A.s, h);
  const float bb = __fsub_rn(t, A.s);
  const float err = __fadd_rn(__fsub_rn(A.s, __fsub_rn(t, bb)), __fsub_rn(h, bb));
  A.s = t;
  A.e += err + l;
}
// A += k * u for a double-float constant k and a double-float value u
PD_D void acc_add_prod(Acc& A, dfc k, float uh, float ul) {
  const float p = __fmul_rn(uh, k.hi);
  float pe = __fmaf_rn(uh, k.hi, -p);
  pe = __fmaf_rn(uh, k.lo, pe);
  pe = __fmaf_rn(ul, k.hi, pe);
  acc_add(A, p, pe);
}
PD_D df acc_val(const Acc& A) { return fast_two_sum(A.s, A.e); }

PD_D K2 k2_of(dfc k) {
  return K2{make_float2(k.hi, k.hi), make_float2(-k.hi, -k.hi), make_float2(-k.lo, -k.lo)};
}

// Global loads of one time row at this thread's column (centre, segment-edge
// x-neighbours, y-neighbours); zeros outside [0, N) or outside the grid.
template <typename V>
struct RowLd {
  V c, l, r, d, u;
};

template <typename V>
PD_D RowLd<V> load_row(const V* U, const FwdArgs& a, const ColGeom& g, int n) {
  RowLd<V> L;
  L.c = L.l = L.r = L.d = L.u = V{};
  if (n >= 0 && n < a.N && g.valid) {
    const size_t base = (size_t)n * a.S;
    L.c = __ldg(&U[base + g.s]);
    if (g.left == 2) L.l = __ldg(&U[base + g.s_left]);
    if (g.right == 2) L.r = __ldg(&U[base + g.s_right]);
    if (g.down) L.d = __ldg(&U[base + g.s - a.st.nx]);
    if (g.up) L.u = __ldg(&U[base + g.s + a.st.nx]);
  }
  return L;
}

// (U(s), (sK U)(s)) in double-float from a loaded row; the x-neighbours of
// interior lanes come from the neighbouring lanes.  Must be executed by all
// lanes of the warp (uniform control flow).
PD_D void stencil_df(const FwdArgs& a, const ColGeom& g, const RowLd<float2>& L, int TX, df& Uc,
                     Acc& KU) {
  const unsigned FULL = 0xffffffffu;
  const float lh = __shfl_up_sync(FULL, L.c.x, 1, TX);
  const float ll = __shfl_up_sync(FULL, L.c.y, 1, TX);
  const float rh = __shfl_down_sync(FULL, L.c.x, 1, TX);
  const float rl = __shfl_down_sync(FULL, L.c.y, 1, TX);
  Uc = df_make(L.c.x, L.c.y);
  // neighbour values: from the lanes beside this one, or the loaded halo / wrap
  // value (zero where the grid has no neighbour), so the sum has no branches
  const bool sl = g.left == 1, sr = g.right == 1;
  Acc A = {0.f, 0.f};
  acc_add_prod(A, a.kap[0], L.c.x, L.c.y);
  acc_add_prod(A, a.kap[1], sl ? lh : L.l.x, sl ? ll : L.l.y);
  acc_add_prod(A, a.kap[2], sr ? rh : L.r.x, sr ? rl : L.r.y);
  if (a.st.dim == 2) {
    acc_add_prod(A, a.kap[3], L.d.x, L.d.y);
    acc_add_prod(A, a.kap[4], L.u.x, L.u.y);
  }
  KU = A;
}

// Packed form of stencil_df: two time rows (lanes A, B) of this thread's column.
template <bool D1 = false>
PD_D void stencil_df2(const FwdArgs& a, const ColGeom& g, const RowLd<float2>& LA,
                      const RowLd<float2>& LB, int TX, const K2* kk, DF2& Uc, Acc2& KU) {
  const unsigned FULL = 0xffffffffu;
  Uc = df2_pack(LA.c, LB.c);
  DF2 lf, rt;
  lf.hi.x = __shfl_up_sync(FULL, Uc.hi.x, 1, TX);
  lf.hi.y = __shfl_up_sync(FULL, Uc.hi.y, 1, TX);
  lf.lo.x = __shfl_up_sync(FULL, Uc.lo.x, 1, TX);
  lf.lo.y = __shfl_up_sync(FULL, Uc.lo.y, 1, TX);
  rt.hi.x = __shfl_down_sync(FULL, Uc.hi.x, 1, TX);
  rt.hi.y = __shfl_down_sync(FULL, Uc.hi.y, 1, TX);
  rt.lo.x = __shfl_down_sync(FULL, Uc.lo.x, 1, TX);
  rt.lo.y = __shfl_down_sync(FULL, Uc.lo.y, 1, TX);
  if (g.left != 1) lf = df2_pack(LA.l, LB.l);
  if (g.right != 1) rt = df2_pack(LA.r, LB.r);
  Acc2 A = acc2_of_prod(kk[0], Uc);
  acc2_add_prod(A, kk[1], lf);
  acc2_add_prod(A, kk[2], rt);
  if (!D1 && a.st.dim == 2) {
    acc2_add_prod(A, kk[3], df2_pack(LA.d, LB.d));
    acc2_add_prod(A, kk[4], df2_pack(LA.u, LB.u));
  }
  KU = A;
}

PD_D void stencil_64(const FwdArgs& a, const ColGeom& g, const RowLd<double>& L, int TX,
                     double& Uc, double& KU) {
  const unsigned FULL = 0xffffffffu;
  const double lv = __shfl_up_sync(FULL, L.c, 1, TX);
  const double rv = __shfl_down_sync(FULL, L.c, 1, TX);
  const Stencil& st = a.st;
  Uc = L.c;
  double k = st.kc * L.c;
  if (g.left == 1) k = fma(st.kxl, lv, k);
  else if (g.left == 2) k = fma(st.kxl, L.l, k);
  if (g.right == 1) k = fma(st.kxu, rv, k);
  else if (g.right == 2) k = fma(st.kxu, L.r, k);
  if (g.down) k = fma(st.kyl, L.d, k);
  if (g.up) k = fma(st.kyu, L.u, k);
  KU = k;
}

template <typename T>
PD_D T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < TT / 32; ++w) s += red[w];
  return s;
}

// ---------------------------------------------------------------------------
// K1: residual (optional) + Gamma scaling + forward real FFT along t.
// PREC 0: mixed (double-float residual, FP32 transform); PREC 1: FP64.
// ---------------------------------------------------------------------------
// D1: 1D problems only (no y-neighbour loads or registers).
// CR > 1: the tile's transform is split over a cluster of CR blocks (power-of-
// two N, see cluster_radix); this block forms the residual of the time rows
// [n_lo, n_lo + N/CR) and writes the spectrum rows k = CR k' + rank.
template <int PREC, int BAND, int EPT, bool D1 = false, int CR = 1>
PD_D void time_fwd_body(const FwdArgs& a, int tile) {
  using R = typename std::conditional<PREC == 0, float, double>::type;
  using C = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  R* smr = reinterpret_cast<R*>(smraw);
  __shared__ double red[TT / 32];

  const int TX = a.TX, N = a.N, S = a.S;
  const int lgTX = ilog2(TX);
  const int x0 = tile * TX;
  const int x = threadIdx.x & (TX - 1);
  // time rows of this block: [n_lo, n_hi), NL of them
  const int rank = CR > 1 ? cluster_rank() : 0;
  const int NL = N / CR, n_lo = rank * NL, n_hi = n_lo + NL;
  // the transform's twiddle table, staged in shared memory after the tile
  // (split transform: the length-NL table W_N^{CR i})
  const int rows_fft = CR > 1 ? NL : (a.xf.M ? a.xf.M : N);
  C* stw = sm + (size_t)rows_fft * (TX / 2);
  for (int i = threadIdx.x; i < rows_fft; i += TT) stw[i] = reinterpret_cast<const C*>(a.tw)[i * CR];
  const int chunk = threadIdx.x >> lgTX;
  const int nchunks = TT / TX;
  const int rpc = (NL + nchunks - 1) / nchunks;
  const int n_beg = n_lo + chunk * rpc;
  const int s = x0 + x;
  const R* gam = reinterpret_cast<const R*>(a.gam);
  double nrm = 0.0;

  // the mode may come from device memory (the solver's graph decides it)
  const int mode = a.mode_dev != nullptr ? *a.mode_dev : a.mode;
  if (mode == FWD_STANDALONE) {
    // every element of the tile: consecutive threads take consecutive columns,
    // eight loads in flight per thread
    constexpr int U = 8;
    const int n0 = threadIdx.x >> lgTX, nstep = TT >> lgTX;
    for (int nb = n0; nb < NL; nb += U * nstep) {
      double rv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int n = nb + u * nstep;
        rv[u] = (n < NL && s < S) ? a.r64[(size_t)(n_lo + n) * S + s] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int n = nb + u * nstep;
        if (n >= NL) break;
        R v;
        if constexpr (PREC == 0) {
          const df r = df_from_double(rv[u]);
          const float gg = gam[n_lo + n];
          v = fmaf(r.hi, gg, r.lo * gg);
        } else {
          v = gam[n_lo + n] * rv[u];
        }
        smr[n * TX + x] = v;
      }
    }
  } else {
    const ColGeom g = col_geom(a.st, s, x, TX);
    if constexpr (PREC == 0) {
      // Two row chunks per thread, computed together in the two lanes of
      // float2 values: lane A rows nA + i, lane B rows nB + i (i < rpc2).
      // Rows before the first level are zero, so the carried terms need no checks.
      const int rpc2 = (NL + 2 * nchunks - 1) / (2 * nchunks);
      const int nA = n_lo + chunk * rpc2, nB = nA + nchunks * rpc2;
      if (mode == FWD_ZERO_GUESS) {
        // r' = s b: the residual loop below with U = 0 (every term it adds to
        // the accumulator is an exact zero), row for row, so the spectrum and
        // the norm are those of FWD_RESIDUAL on a zero iterate
        const int Nm1 = N - 1;
        const float2* __restrict__ Bcol = a.Bdf + (g.valid ? s : 0);
        float2 part = make_float2(0.f, 0.f);
        float* srow = smr + x;
#pragma unroll 4
        for (int i = 0; i < rpc2; ++i) {
          const int na = nA + i, nb = nB + i;
          const float2 bA = __ldg(Bcol + (size_t)min(na, Nm1) * S);
          const float2 bB = __ldg(Bcol + (size_t)min(nb, Nm1) * S);
          const DF2 Bv = df2_pack(bA, bB);
          const float2 rh = f2add(Bv.hi, Bv.lo);
          const float2 rl = f2sub(Bv.lo, f2sub(rh, Bv.hi));
          const bool va = na < n_hi && g.valid, vb = nb < n_hi && g.valid;
          const float2 rn = make_float2(va ? rh.x : 0.f, vb ? rh.y : 0.f);
          part = f2fma(rn, rn, part);
          if (na < n_hi) srow[(na - n_lo) * TX] = va ? fmaf(rh.x, gam[na], rl.x * gam[na]) : 0.f;
          if (nb < n_hi) srow[(nb - n_lo) * TX] = vb ? fmaf(rh.y, gam[nb], rl.y * gam[nb]) : 0.f;
        }
        const float part1 = part.x + part.y;
        nrm = (double)part1 * a.rscale2;
      } else {
      K2 kk[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) kk[q] = k2_of(a.kap[q]);
      DF2 U1 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, U2 = U1, U0;
      Acc2 K1 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, K2v = K1, K0;
      if (BAND == 2)
        stencil_df2<D1>(a, g, load_row(a.Udf, a, g, nA - 2), load_row(a.Udf, a, g, nB - 2), TX, kk,
                    U2, K2v);
      stencil_df2<D1>(a, g, load_row(a.Udf, a, g, nA - 1), load_row(a.Udf, a, g, nB - 1), TX, kk, U1,
                  K1);
      // In the loop every row index is clamped to the last level: rows at or
      // past N (possible in the last chunks) are computed from in-range data
      // and discarded, so the loads carry no row checks.  Padding columns
      // (s >= S) read column 0 and write zeros; no valid column takes an
      // x-neighbour from a padding lane (the last grid point has none to its
      // right, or a wrapped one that is loaded).
      const int sc = g.valid ? s : 0;
      const bool hasL = g.left == 2, hasR = g.right == 2, hasD = g.down, hasU = g.up;
      const int dL = hasL ? g.s_left - s : 0, dR = hasR ? g.s_right - s : 0;
      const int nx = a.st.nx, Nm1 = N - 1;
      const size_t Sz = (size_t)S;
      const float2* __restrict__ Ucol = a.Udf + sc;
      const float2* __restrict__ Bcol = a.Bdf + sc;
      const float2 z2 = make_float2(0.f, 0.f);
      auto ldrow = [&](int n) -> RowLd<float2> {
        const float2* p = Ucol + (size_t)n * Sz;
        RowLd<float2> L;
        L.c = __ldg(p);
        L.l = hasL ? __ldg(p + dL) : z2;
        L.r = hasR ? __ldg(p + dR) : z2;
        L.d = (!D1 && hasD) ? __ldg(p - nx) : z2;
        L.u = (!D1 && hasU) ? __ldg(p + nx) : z2;
        return L;
      };
      // one row of loads in flight ahead of the row being computed
      RowLd<float2> cA = ldrow(min(nA, Nm1)), cB = ldrow(min(nB, Nm1));
      float2 bA = __ldg(Bcol + (size_t)min(nA, Nm1) * Sz);
      float2 bB = __ldg(Bcol + (size_t)min(nB, Nm1) * Sz);
      // the c2 weights negated once; when every c2[m] is 0 or a power of two
      // (backward Euler, Crank-Nicolson, leap-frog) the weighted terms are exact
      // scalings
      dfc m0 = a.e2[0], mb = BAND == 1 ? a.e2[1] : a.e2[2];
      m0.hi = -m0.hi; m0.lo = -m0.lo;
      mb.hi = -mb.hi; mb.lo = -mb.lo;
      const bool exact = a.c2exact != 0;
      const bool has_mb = mb.hi != 0.f;
      const K2 km0 = k2_of(m0), kmb = k2_of(mb);
      const float2 sm0 = make_float2(m0.hi, m0.hi), smb = make_float2(mb.hi, mb.hi);
      const float2 two = make_float2(2.f, 2.f);
      float2 part = make_float2(0.f, 0.f);
      float* srow = smr + x;
#pragma unroll 1
      for (int i = 0; i < rpc2; ++i) {
        const int na = nA + i, nb = nB + i;
        const int pa = min(na + 1, Nm1), pb = min(nb + 1, Nm1);
        const RowLd<float2> xA = ldrow(pa), xB = ldrow(pb);
        const float2 yA = __ldg(Bcol + (size_t)pa * Sz), yB = __ldg(Bcol + (size_t)pb * Sz);
        stencil_df2<D1>(a, g, cA, cB, TX, kk, U0, K0);  // uniform across the warp
        // r' = s b - U_n + U_{n-1} - c2[0] (sK)U_n - c2[1] (sK)U_{n-1}        (theta)
        // r' = s b - U_n + 2 U_{n-1} - U_{n-2} - c2[0] (sK)U_n - c2[2] (sK)U_{n-2} (leap-frog)
        const DF2 Bv = df2_pack(bA, bB);
        Acc2 A = {Bv.hi, Bv.lo};
        acc2_sub(A, U0.hi, U0.lo);
        if (BAND == 1) {
          acc2_add(A, U1.hi, U1.lo);
        } else {
          acc2_add(A, f2mul(two, U1.hi), f2mul(two, U1.lo));
          acc2_sub(A, U2.hi, U2.lo);
        }
        const Acc2& Kb = BAND == 1 ? K1 : K2v;
        if (exact) {
          acc2_add(A, f2mul(sm0, K0.s), f2mul(sm0, K0.e));
          if (has_mb) acc2_add(A, f2mul(smb, Kb.s), f2mul(smb, Kb.e));
        } else {
          acc2_add_prod(A, km0, DF2{K0.s, K0.e});
          acc2_add_prod(A, kmb, DF2{Kb.s, Kb.e});
        }
        // value = s + e, renormalised
        const float2 rh = f2add(A.s, A.e);
        const float2 rl = f2sub(A.e, f2sub(rh, A.s));
        // rows at or past n_hi (lanes of the last chunks) add nothing
        const bool va = na < n_hi && g.valid, vb = nb < n_hi && g.valid;
        const float2 rn = make_float2(va ? rh.x : 0.f, vb ? rh.y : 0.f);
        part = f2fma(rn, rn, part);
        if (na < n_hi) {
          const float gg = gam[na];
          srow[(na - n_lo) * TX] = va ? fmaf(rh.x, gg, rl.x * gg) : 0.f;
        }
        if (nb < n_hi) {
          const float gg = gam[nb];
          srow[(nb - n_lo) * TX] = vb ? fmaf(rh.y, gg, rl.y * gg) : 0.f;
        }
        U2 = U1; K2v = K1; U1 = U0; K1 = K0;
        cA = xA; cB = xB;
        bA = yA; bB = yB;
      }
      const float part1 = part.x + part.y;
      nrm = (double)part1 * a.rscale2;
      }
    } else {
      double U1 = 0, U2 = 0, K1 = 0, K2 = 0, U0, K0;
      const TimeBand& tb = a.tb;
      if (BAND == 2) stencil_64(a, g, load_row(a.U64, a, g, n_beg - 2), TX, U2, K2);
      stencil_64(a, g, load_row(a.U64, a, g, n_beg - 1), TX, U1, K1);
      RowLd<double> cur = load_row(a.U64, a, g, n_beg);
      double bcur = (n_beg < N && g.valid) ? __ldg(&a.B64[(size_t)n_beg * S + s]) : 0.0;
      for (int i = 0; i < rpc; ++i) {
        const int n = n_beg + i;
        const RowLd<double> nxt = load_row(a.U64, a, g, i + 1 < rpc ? n + 1 : -1);
        const double bnxt = (i + 1 < rpc && n + 1 < N && g.valid)
                                ? __ldg(&a.B64[(size_t)(n + 1) * S + s]) : 0.0;
        stencil_64(a, g, cur, TX, U0, K0);
        if (n < n_hi) {
          double v = 0.0;
          if (g.valid) {
            double r = bcur;
            r = fma(-tb.c1[0], U0, r);
            r = fma(-tb.c2[0], K0, r);
            if (n >= 1) { r = fma(-tb.c1[1], U1, r); r = fma(-tb.c2[1], K1, r); }
            if (BAND == 2 && n >= 2) { r = fma(-tb.c1[2], U2, r); r = fma(-tb.c2[2], K2, r); }
            nrm = fma(r, r, nrm);
            v = gam[n] * r;
          }
          smr[(n - n_lo) * TX + x] = v;
        }
        U2 = U1; K2 = K1; U1 = U0; K1 = K0;
        cur = nxt;
        bcur = bnxt;
      }
    }
  }
  if (a.norm2 != nullptr) {
    const double bs = block_sum<double>(nrm, red);
    if (threadIdx.x == 0) atomicAdd(a.norm2, bs);
  }
  if (mode == FWD_RESIDUAL_NORM) return;  // uniform across the block
  __syncthreads();

  const int lgTXc = lgTX - 1;
  const int TXc = TX / 2;
  if constexpr (CR > 1) {
    // the radix-CR step over the cluster, then this block's length-NL part
    cluster_sync();
    cluster_radix<C, false, CR>(sm, NL, lgTXc, reinterpret_cast<const C*>(a.tw), rank);
    cluster_sync();
    fft_tile<C, false, EPT>(sm, NL, a.logN - ilog2(CR), lgTXc, stw);
    cluster_sync();   // every block's spectrum rows, for the partner reads below
  } else {
    if (a.xf.M == 0) fft_tile<C, false, EPT>(sm, N, a.logN, lgTXc, stw);
    else bluestein_tile<C, false, EPT>(sm, N, a.xf, lgTXc, stw);
  }

  C* out = reinterpret_cast<C*>(a.out);
  const R half = (R)0.5;
  {
    // TT is a multiple of TXc: every item of this thread has the same column
    // pair, so the (padded) spectrum offsets are computed once
    const int c = threadIdx.x & (TXc - 1);
    const int sa = x0 + 2 * c;
    const bool va = sa < S, vb = sa + 1 < S;
    const size_t oa = va ? spec_index(a.sg, 0, sa) : 0;
    const size_t ob = vb ? spec_index(a.sg, 0, sa + 1) : 0;
    const size_t kst = (size_t)a.sg.specS;
    R mx = 0;
    if constexpr (CR > 1) {
      // row k' of this block is Z_k, k = CR k' + rank; Z_{N-k} is row
      // (NL - k') mod NL of block 0 (rank 0) or row NL - 1 - k' of block CR - rank
      const uint32_t pb = dsm_map(sm, rank == 0 ? 0 : CR - rank);
      for (int kp = threadIdx.x >> lgTXc; CR * kp + rank < a.nh; kp += TT >> lgTXc) {
        const int k = CR * kp + rank;
        const int pr = rank == 0 ? ((NL - kp) & (NL - 1)) : NL - 1 - kp;
        const C Zk = sm[(kp << lgTXc) + c];
        const C Zm = cconj(dsm_ld(pb + (uint32_t)(((pr << lgTXc) + c) * (int)sizeof(C)), C{}));
        const C A = cscale(cadd(Zk, Zm), half);
        const C B = cscale(cmul_mi(csub(Zk, Zm)), half);
        if (va) out[k * kst + oa] = A;
        if (vb) out[k * kst + ob] = B;
        mx = fmax(mx, fmax(fmax(fabs(A.x), fabs(A.y)), fmax(fabs(B.x), fabs(B.y))));
      }
      cluster_sync();   // no block leaves while its rows may still be read
    } else {
      for (int k = threadIdx.x >> lgTXc; k < a.nh; k += TT >> lgTXc) {
        const C Zk = sm[(k << lgTXc) + c];
        const C Zm = cconj(sm[((k == 0 ? 0 : N - k) << lgTXc) + c]);
        const C A = cscale(cadd(Zk, Zm), half);
        const C B = cscale(cmul_mi(csub(Zk, Zm)), half);
        if (va) out[k * kst + oa] = A;
        if (vb) out[k * kst + ob] = B;
        mx = fmax(mx, fmax(fmax(fabs(A.x), fabs(A.y)), fmax(fabs(B.x), fabs(B.y))));
      }
    }
    if constexpr (PREC == 0) {
      // largest |value| for the scaling of the tensor-core x-transform
      if (a.amax != nullptr) {
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) atomicMax(a.amax, __float_as_uint(mx));
        if (a.amax_reset != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *a.amax_reset = 0u;
      }
    }
  }
}

// single problem: block b owns tile b; batch: the work table maps each block to
// (problem, tile) and the arguments come from the per-problem descriptors
template <int PREC, int BAND, int EPT>
__global__ void __launch_bounds__(TT, PREC == 0 ? 3 : 2) k_time_fwd(FwdArgs a) {
  time_fwd_body<PREC, BAND, EPT>(a, blockIdx.x);
}
// a tile per cluster of CR blocks (the transform split as in cluster_radix)
// (D1: 1D problems, no y-neighbour registers)
template <int PREC, int BAND, int EPT, int CR, bool D1>
__global__ void __cluster_dims__(CR, 1, 1) __launch_bounds__(TT, PREC == 0 ? 3 : 2)
    k_time_fwd_cl(FwdArgs a) {
  time_fwd_body<PREC, BAND, EPT, D1, CR>(a, blockIdx.x / CR);
}
// batch: one block per entry of the work table (problem, tile).  A persistent
// form (blocks taking entries from a device counter) was measured slower for
// these kernels (forward 0.70 against 0.57 ms, inverse 0.51 against 0.35 ms
// per sweep of the 64-problem batch), so the hardware block scheduler assigns
// the tiles.
template <int PREC, int BAND, int EPT>
__global__ void __launch_bounds__(TT, PREC == 0 ? 3 : 2) k_time_fwd_batch(const FwdArgs* __restrict__ descs,
                                                          const int2* __restrict__ work) {
  const int2 w = work[blockIdx.x];
  // batches hold 1D problems only
  time_fwd_body<PREC, BAND, EPT, true>(descs[w.x], w.y);
}

// ---------------------------------------------------------------------------
// K3: inverse real FFT along t + Gamma^{-1}/Nt + write or update.
// ---------------------------------------------------------------------------
// CR > 1: the transform is split over a cluster of CR blocks (power-of-two N,
// see cluster_radix); this block reads the spectrum rows k = CR k' + rank (or
// their mirrors N - k) and writes the time rows [n_lo, n_lo + N/CR).
template <int PREC, int EPT, int CR = 1>
PD_D void time_inv_body(const InvArgs& a, int tile) {
  using R = typename std::conditional<PREC == 0, float, double>::type;
  using C = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  R* smr = reinterpret_cast<R*>(smraw);

  const int TX = a.TX, N = a.N, S = a.S;
  const int lgTX = ilog2(TX), lgTXc = lgTX - 1, TXc = TX / 2;
  const int x0 = tile * TX;
  const int rank = CR > 1 ? cluster_rank() : 0;
  const int NL = N / CR, n_lo = rank * NL;
  const C* in = reinterpret_cast<const C*>(a.in);
  const int rows_fft = CR > 1 ? NL : (a.xf.M ? a.xf.M : N);
  C* stw = sm + (size_t)rows_fft * TXc;
  for (int i = threadIdx.x; i < rows_fft; i += TT) stw[i] = reinterpret_cast<const C*>(a.tw)[i * CR];
  if constexpr (CR > 1) {
    // Z_k = A_k + i B_k for k = CR k' + rank; past N/2 from the mirror row
    // N - k: Z_k = conj(A_{N-k}) + i conj(B_{N-k})
    const int c = threadIdx.x & (TXc - 1);
    const int sa = x0 + 2 * c;
    const bool va = sa < S, vb = sa + 1 < S;
    const size_t oa = va ? spec_index(a.sg, 0, sa) : 0;
    const size_t ob = vb ? spec_index(a.sg, 0, sa + 1) : 0;
    const size_t kst = (size_t)a.sg.specS;
    const int k0 = threadIdx.x >> lgTXc, kstep = TT >> lgTXc;
    constexpr int U = 8;  // loads in flight per thread
    for (int kb = k0; kb < NL; kb += U * kstep) {
      C A[U], B[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kp = kb + u * kstep;
        const int k = CR * kp + rank;
        const int kr = k < a.nh ? k : N - k;
        A[u] = czero<C>();
        B[u] = czero<C>();
        if (kp < NL) {
          if (va) A[u] = in[kr * kst + oa];
          if (vb) B[u] = in[kr * kst + ob];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kp = kb + u * kstep;
        if (kp >= NL) break;
        const int k = CR * kp + rank;
        C Au = A[u], Bu = B[u];
        if (k == 0 || 2 * k == N) { Au.y = 0; Bu.y = 0; }
        sm[(kp << lgTXc) + c] = k < a.nh ? mk(Au.x - Bu.y, Au.y + Bu.x)   // A + i B
                                         : mk(Au.x + Bu.y, Bu.x - Au.y);  // conj(A) + i conj(B)
      }
    }
  } else {
    const int c = threadIdx.x & (TXc - 1);
    const int sa = x0 + 2 * c;
    const bool va = sa < S, vb = sa + 1 < S;
    const size_t oa = va ? spec_index(a.sg, 0, sa) : 0;
    const size_t ob = vb ? spec_index(a.sg, 0, sa + 1) : 0;
    const size_t kst = (size_t)a.sg.specS;
    const int k0 = threadIdx.x >> lgTXc, kstep = TT >> lgTXc;
    constexpr int U = 8;  // loads in flight per thread
    for (int kb = k0; kb < a.nh; kb += U * kstep) {
      C A[U], B[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = kb + u * kstep;
        A[u] = czero<C>();
        B[u] = czero<C>();
        if (k < a.nh) {
          if (va) A[u] = in[k * kst + oa];
          if (vb) B[u] = in[k * kst + ob];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = kb + u * kstep;
        if (k >= a.nh) break;
        C Au = A[u], Bu = B[u];
        if (k == 0 || 2 * k == N) { Au.y = 0; Bu.y = 0; }
        sm[(k << lgTXc) + c] = mk(Au.x - Bu.y, Au.y + Bu.x);            // A + i B
        if (k > 0 && 2 * k < N)
          sm[((N - k) << lgTXc) + c] = mk(Au.x + Bu.y, Bu.x - Au.y);    // conj(A) + i conj(B)
      }
    }
  }
  __syncthreads();
  if constexpr (CR > 1) {
    fft_tile<C, true, EPT>(sm, NL, a.logN - ilog2(CR), lgTXc, stw);
    cluster_sync();
    cluster_radix<C, true, CR>(sm, NL, lgTXc, reinterpret_cast<const C*>(a.tw), rank);
    cluster_sync();
  } else {
    if (a.xf.M == 0) fft_tile<C, true, EPT>(sm, N, a.logN, lgTXc, stw);
    else bluestein_tile<C, true, EPT>(sm, N, a.xf, lgTXc, stw);
  }

  const R* ig = reinterpret_cast<const R*>(a.igam);
  // the mode may come from device memory (the solver's graph decides it)
  const int mode = a.mode_dev != nullptr ? *a.mode_dev : a.mode;
  bool bad = false;
  {
    // every element of this thread lies in the same column x (TT % TX == 0)
    const int x = threadIdx.x & (TX - 1);
    const int s = x0 + x;
    const int n0 = threadIdx.x >> lgTX, nstep = TT >> lgTX;
    constexpr int U = 8;
    if (s < S) {
      for (int nb = n0; nb < NL; nb += U * nstep) {
        if constexpr (PREC == 0) {
          float2 uv[U];
          if (mode == INV_UPDATE_DF) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int n = nb + u * nstep;
              uv[u] = n < NL ? a.Udf[(size_t)(n_lo + n) * S + s] : make_float2(0.f, 0.f);
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int n = nb + u * nstep;   // row n_lo + n
            if (n >= NL) break;
            const float dz = smr[n * TX + x] * ig[n_lo + n];
            if (!isfinite(dz)) bad = true;
            const size_t idx = (size_t)(n_lo + n) * S + s;
            if (mode == INV_UPDATE_DF) {
              df t = two_sum(uv[u].x, dz);
              t = fast_two_sum(t.hi, t.lo + uv[u].y);
              a.Udf[idx] = make_float2(t.hi, t.lo);
            } else if (mode == INV_SET_DF) {
              a.Udf[idx] = make_float2(dz, 0.f);
            } else {
              a.out64[idx] = double_from_float(dz);
            }
          }
        } else {
          double uv[U];
          if (mode == INV_UPDATE64) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int n = nb + u * nstep;
              uv[u] = n < NL ? a.out64[(size_t)(n_lo + n) * S + s] : 0.0;
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int n = nb + u * nstep;   // row n_lo + n
            if (n >= NL) break;
            const double dz = smr[n * TX + x] * ig[n_lo + n];
            if (!isfinite(dz)) bad = true;
            const size_t idx = (size_t)(n_lo + n) * S + s;
            a.out64[idx] = (mode == INV_UPDATE64) ? uv[u] + dz : dz;
          }
        }
      }
    }
  }
  if (bad && a.flag != nullptr) atomicOr(a.flag, 1);
}

template <int PREC, int EPT>
__global__ void __launch_bounds__(TT, PREC == 0 ? 4 : 2) k_time_inv(InvArgs a) {
  time_inv_body<PREC, EPT>(a, blockIdx.x);
}
template <int PREC, int EPT, int CR>
__global__ void __cluster_dims__(CR, 1, 1) __launch_bounds__(TT, PREC == 0 ? 4 : 2)
    k_time_inv_cl(InvArgs a) {
  time_inv_body<PREC, EPT, CR>(a, blockIdx.x / CR);
}
template <int PREC, int EPT>
__global__ void __launch_bounds__(TT, PREC == 0 ? 4 : 2) k_time_inv_batch(const InvArgs* __restrict__ descs,
                                                         const int2* __restrict__ work) {
  const int2 w = work[blockIdx.x];
  time_inv_body<PREC, EPT>(descs[w.x], w.y);
}

// ---------------------------------------------------------------------------
// x-eigentransform by FFT (step (b) of 2D problems and of periodic 1D
// problems; FP64 on FP64 plans, FP32 on mixed plans, where it competes with the
// tensor-core GEMM): every row of the half spectrum is transformed along
// x by the DFT (periodic x: the eigenvectors of the circulant K_x) or by the
// sine transform (symmetric Dirichlet x), in O(nx log nx) instead of the dense
// O(nx^2) product.  A block holds XR rows transposed in shared memory (element
// m of row r at m XR + r, the layout of the time kernels' tiles) and runs the
// same Stockham / Bluestein routines on them.
//   periodic, forward: Y_j = sum_x X_x e^{-2 pi i j x / nx}
//   periodic, inverse: X_x = (1/nx) sum_j Y_j e^{+2 pi i j x / nx}
//   sine transform:    Y_j = sum_x sin(pi (j+1)(x+1)/(nx+1)) X_x
//                          = (i/2) V_{j+1}, V the length-2(nx+1) DFT of the odd
//                            extension v = (0, X, 0, -X reversed);
//                      the inverse is the same transform times 2/(nx+1).
// ---------------------------------------------------------------------------
constexpr int XR = 4;   // rows per block

template <typename C, int EPT>
__global__ void __launch_bounds__(TT) k_xform_fft(XfftArgs a) {
  using R = decltype(C::x);
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const int rows_fft = a.xf.M ? a.xf.M : a.L;
  C* stw = sm + (size_t)rows_fft * XR;
  for (int i = threadIdx.x; i < rows_fft; i += TT) stw[i] = reinterpret_cast<const C*>(a.tw)[i];
  const int r0 = blockIdx.x * XR;
  const C* in = reinterpret_cast<const C*>(a.in);
  C* out = reinterpret_cast<C*>(a.out);
  const int L = a.L, nx = a.nx;
  // input rows (zero rows past the end), transposed into the tile
  for (int e = threadIdx.x; e < XR * L; e += TT) {
    const int r = e / L, m = e - r * L;
    const int row = r0 + r;
    C v = czero<C>();
    if (row < a.rows) {
      if (!a.dst) {
        v = in[(size_t)row * a.ld + m];
      } else if (m >= 1 && m <= nx) {
        v = in[(size_t)row * a.ld + (m - 1)];                     // v_{x+1} = X_x
      } else if (m >= nx + 2) {
        const C w = in[(size_t)row * a.ld + (L - 1 - m)];         // v_{L-1-x} = -X_x
        v = mk(-w.x, -w.y);
      }
    }
    sm[m * XR + r] = v;
  }
  __syncthreads();
  constexpr int lgXR = 2;
  const bool inv = a.inv != 0 && !a.dst;                         // the sine transform is its own kind
  if (a.xf.M == 0) {
    if (inv) fft_tile<C, true, EPT>(sm, L, a.logL, lgXR, stw);
    else fft_tile<C, false, EPT>(sm, L, a.logL, lgXR, stw);
  } else {
    if (inv) bluestein_tile<C, true, EPT>(sm, L, a.xf, lgXR, stw);
    else bluestein_tile<C, false, EPT>(sm, L, a.xf, lgXR, stw);
  }
  // outputs
  const R sc = (R)(a.dst ? (a.inv ? 1.0 / (nx + 1) : 0.5) : (a.inv ? 1.0 / nx : 1.0));
  for (int e = threadIdx.x; e < XR * nx; e += TT) {
    const int r = e / nx, j = e - r * nx;
    const int row = r0 + r;
    if (row >= a.rows) continue;
    C y;
    if (!a.dst) {
      y = sm[j * XR + r];
      y = mk(y.x * sc, y.y * sc);
    } else {
      const C v = sm[(j + 1) * XR + r];                          // (i/2) V_{j+1}, scaled
      y = mk(-v.y * sc, v.x * sc);
    }
    out[(size_t)row * a.ld + j] = y;
  }
}

template <typename C, int EPT>
cudaError_t launch_xfft_e(const XfftArgs& a, cudaStream_t st) {
  const int rows_fft = a.xf.M ? a.xf.M : a.L;
  const size_t smem = (size_t)rows_fft * (XR + 1) * sizeof(C);
  auto kern = k_xform_fft<C, EPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<ceil_div(a.rows, XR), TT, smem, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The same transforms for lengths L = L1 L2 with both factors at most 32 and L
// not a power of two (periodic nx = 255 = 15 x 17, for one): one Cooley-Tukey
// step with two direct DFTs instead of Bluestein's two length-M FFTs.  With
// n = L2 n1 + n2 and j = k1 + L1 k2,
//   X_j = sum_{n2} W_{L2}^{n2 k2} [ W_L^{n2 k1} sum_{n1} x_{L2 n1 + n2} W_{L1}^{n1 k1} ],
// W_m = exp(-2 pi i / m) (the conjugate root for the inverse).  A block holds
// XB = 256 / L2 rows in shared memory, [row][L].  Step 1: item (row, n2) sums
// its L1 inputs (stride L2) into L1 accumulators, applies W_L^{n2 k1} and
// writes them back to the positions it read, L2 k1 + n2 (so the step runs in
// place).  Step 2: item (row, k1) sums the L2 contiguous values of its group
// into L2 accumulators and stores X_{k1 + L1 k2} (scaled; for the sine
// transform the odd extension's entries 1..nx) to global memory.  B >= L1, L2
// bounds the accumulator arrays at compile time.  Every twiddle is an entry
// of the length-L table W_L^m, m < L, held in shared memory; the index of
// W_{L1}^{n1 k1} = W_L^{L2 (n1 k1 mod L1)} steps by n1 L2 modulo L.
// ---------------------------------------------------------------------------
template <typename C, int B>
__global__ void __launch_bounds__(TT) k_xform_dft2(XfftArgs a) {
  using R = decltype(C::x);
  extern __shared__ __align__(16) unsigned char smraw[];
  const int L = a.L, L1 = a.L1, L2 = a.L2, nx = a.nx;
  const int XB = TT / L2;
  C* sm = reinterpret_cast<C*>(smraw);          // [XB][L]
  C* stw = sm + (size_t)XB * L;                 // W_L^m, m < L
  for (int i = threadIdx.x; i < L; i += TT) stw[i] = reinterpret_cast<const C*>(a.tw)[i];
  const int r0 = blockIdx.x * XB;
  const C* in = reinterpret_cast<const C*>(a.in);
  C* out = reinterpret_cast<C*>(a.out);
  // input rows (zero rows past the end; the sine transform's odd extension)
  for (int e = threadIdx.x; e < XB * L; e += TT) {
    const int r = e / L, m = e - r * L;
    const int row = r0 + r;
    C v = czero<C>();
    if (row < a.rows) {
      if (!a.dst) {
        v = in[(size_t)row * a.ld + m];
      } else if (m >= 1 && m <= nx) {
        v = in[(size_t)row * a.ld + (m - 1)];                     // v_{x+1} = X_x
      } else if (m >= nx + 2) {
        const C w = in[(size_t)row * a.ld + (L - 1 - m)];         // v_{L-1-x} = -X_x
        v = mk(-w.x, -w.y);
      }
    }
    sm[e] = v;
  }
  __syncthreads();
  const bool inv = a.inv != 0 && !a.dst;
  auto tw_at = [&](int m) -> C {
    C w = stw[m];
    if (inv) w.y = -w.y;
    return w;
  };
  // step 1: length-L1 DFTs over n1, then the twiddle W_L^{n2 k1}
  {
    const int item = threadIdx.x;
    if (item < XB * L2) {
      const int r = item / L2, n2 = item - r * L2;
      C* row = sm + (size_t)r * L;
      C acc[B];
#pragma unroll
      for (int k = 0; k < B; ++k) acc[k] = czero<C>();
      for (int n1 = 0; n1 < L1; ++n1) {
        const C x = row[L2 * n1 + n2];
        const int step = n1 * L2;
        int q = 0;
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (k < L1) {
            const C w = tw_at(q);
            acc[k].x = fma(x.x, w.x, fma(-x.y, w.y, acc[k].x));
            acc[k].y = fma(x.x, w.y, fma(x.y, w.x, acc[k].y));
            q += step;
            if (q >= L) q -= L;
          }
        }
      }
      int q = 0;
#pragma unroll
      for (int k = 0; k < B; ++k) {
        if (k < L1) {
          row[L2 * k + n2] = cmul(acc[k], tw_at(q));
          q += n2;
        }
      }
    }
  }
  __syncthreads();
  // step 2: length-L2 DFTs over n2, outputs j = k1 + L1 k2
  {
    const R sc = (R)(a.dst ? (a.inv ? 1.0 / (nx + 1) : 0.5) : (a.inv ? 1.0 / nx : 1.0));
    const int item = threadIdx.x;
    if (item < XB * L1) {
      const int r = item / L1, k1 = item - r * L1;
      const int row = r0 + r;
      const C* grp = sm + (size_t)r * L + (size_t)L2 * k1;
      C acc[B];
#pragma unroll
      for (int k = 0; k < B; ++k) acc[k] = czero<C>();
      for (int n2 = 0; n2 < L2; ++n2) {
        const C y = grp[n2];
        const int step = n2 * L1;
        int q = 0;
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (k < L2) {
            const C w = tw_at(q);
            acc[k].x = fma(y.x, w.x, fma(-y.y, w.y, acc[k].x));
            acc[k].y = fma(y.x, w.y, fma(y.y, w.x, acc[k].y));
            q += step;
            if (q >= L) q -= L;
          }
        }
      }
      if (row < a.rows) {
        C* orow = out + (size_t)row * a.ld;
#pragma unroll
        for (int k = 0; k < B; ++k) {
          if (k < L2) {
            const int j = k1 + L1 * k;
            if (!a.dst) {
              if (j < nx) orow[j] = mk(acc[k].x * sc, acc[k].y * sc);
            } else if (j >= 1 && j <= nx) {
              orow[j - 1] = mk(-acc[k].y * sc, acc[k].x * sc);     // (i/2) V_j, scaled
            }
          }
        }
      }
    }
  }
}

// The same two steps with the factors fixed at compile time, FP32 (the loops
// fully unrolled, every twiddle index W_{L1}^{(n1 k) mod L1} a constant) and RPI
// rows per item, so that one twiddle load serves RPI complex products.  FP32:
// the table holds (Re w, Im w, Im w, Re w) per entry and a product takes two
// paired FMAs, (x.re, x.re) (Re w, Im w) + (-x.im, x.im) (Im w, Re w).
template <typename C> struct TwS;
template <> struct TwS<float2> { using T = float4; };
template <> struct TwS<double2> { using T = double2; };

PD_D void cmac_tw(float2& acc, const float2& xa, const float2& xb, const float4& w) {
  acc = f2fma(xa, make_float2(w.x, w.y), acc);
  acc = f2fma(xb, make_float2(w.z, w.w), acc);
}
PD_D void cmac_tw(double2& acc, const double2& x, const double2&, const double2& w) {
  acc.x = fma(x.x, w.x, fma(-x.y, w.y, acc.x));
  acc.y = fma(x.x, w.y, fma(x.y, w.x, acc.y));
}
PD_D void cmac_split(const float2& x, float2& xa, float2& xb) {
  xa = make_float2(x.x, x.x);
  xb = make_float2(-x.y, x.y);
}
PD_D void cmac_split(const double2& x, double2& xa, double2& xb) { xa = x; xb = x; }
PD_D float2 tw_c(const float4& w) { return make_float2(w.x, w.y); }
PD_D double2 tw_c(const double2& w) { return w; }

// (three blocks per SM for FP32, 80 registers)
template <typename C, int L1, int L2, int RPI>
__global__ void __launch_bounds__(TT, sizeof(C) == 8 ? 3 : 2) k_xform_dft2r(XfftArgs a) {
  using R = decltype(C::x);
  using T = typename TwS<C>::T;
  constexpr int L = L1 * L2;
  constexpr int NI = TT / L2;            // row groups per block
  constexpr int XB = NI * RPI;           // rows per block
  extern __shared__ __align__(16) unsigned char smraw[];
  T* stw = reinterpret_cast<T*>(smraw);                  // W_L^m (conjugated for the inverse)
  C* stp = reinterpret_cast<C*>(stw + L);                // [k][n2]: W_L^{n2 k}, the step-1 twiddle
  C* sm = stp + L;                                       // [XB][L]
  const int nx = a.nx;
  const bool inv = a.inv != 0 && !a.dst;
  for (int i = threadIdx.x; i < L; i += TT) {
    C w = reinterpret_cast<const C*>(a.tw)[i];
    if (inv) w.y = -w.y;
    if constexpr (sizeof(T) == 16 && sizeof(C) == 8) stw[i] = make_float4(w.x, w.y, w.y, w.x);
    else stw[i] = w;
    // laid out so that the threads of a step-1 store (consecutive n2) read
    // consecutive entries
    const int k = i / L2, n2 = i - k * L2;
    C v = reinterpret_cast<const C*>(a.tw)[n2 * k];
    if (inv) v.y = -v.y;
    stp[i] = v;
  }
  const int r0 = blockIdx.x * XB;
  const C* in = reinterpret_cast<const C*>(a.in);
  C* out = reinterpret_cast<C*>(a.out);
  for (int e = threadIdx.x; e < XB * L; e += TT) {
    const int r = e / L, m = e - r * L;
    const int row = r0 + r;
    C v = czero<C>();
    if (row < a.rows) {
      if (!a.dst) {
        v = in[(size_t)row * a.ld + m];
      } else if (m >= 1 && m <= nx) {
        v = in[(size_t)row * a.ld + (m - 1)];
      } else if (m >= nx + 2) {
        const C w = in[(size_t)row * a.ld + (L - 1 - m)];
        v = mk(-w.x, -w.y);
      }
    }
    sm[e] = v;
  }
  __syncthreads();
  // step 1: item (group g, n2) over the rows g RPI + i
  if (threadIdx.x < NI * L2) {
    const int g = threadIdx.x / L2, n2 = threadIdx.x - g * L2;
    C acc[RPI][L1];
#pragma unroll
    for (int i = 0; i < RPI; ++i)
#pragma unroll
      for (int k = 0; k < L1; ++k) acc[i][k] = czero<C>();
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) {
      C xa[RPI], xb[RPI];
#pragma unroll
      for (int i = 0; i < RPI; ++i)
        cmac_split(sm[(size_t)(g * RPI + i) * L + L2 * n1 + n2], xa[i], xb[i]);
#pragma unroll
      for (int k = 0; k < L1; ++k) {
        const T w = stw[L2 * ((n1 * k) % L1)];
#pragma unroll
        for (int i = 0; i < RPI; ++i) cmac_tw(acc[i][k], xa[i], xb[i], w);
      }
    }
#pragma unroll
    for (int k = 0; k < L1; ++k) {
      const C w = stp[k * L2 + n2];
#pragma unroll
      for (int i = 0; i < RPI; ++i)
        sm[(size_t)(g * RPI + i) * L + L2 * k + n2] = cmul(acc[i][k], w);
    }
  }
  __syncthreads();
  // step 2: item (group g, k1): outputs j = k1 + L1 k2
  if (threadIdx.x < NI * L1) {
    const int g = threadIdx.x / L1, k1 = threadIdx.x - g * L1;
    C acc[RPI][L2];
#pragma unroll
    for (int i = 0; i < RPI; ++i)
#pragma unroll
      for (int k = 0; k < L2; ++k) acc[i][k] = czero<C>();
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) {
      C xa[RPI], xb[RPI];
#pragma unroll
      for (int i = 0; i < RPI; ++i)
        cmac_split(sm[(size_t)(g * RPI + i) * L + L2 * k1 + n2], xa[i], xb[i]);
#pragma unroll
      for (int k = 0; k < L2; ++k) {
        const T w = stw[L1 * ((n2 * k) % L2)];
#pragma unroll
        for (int i = 0; i < RPI; ++i) cmac_tw(acc[i][k], xa[i], xb[i], w);
      }
    }
    const R sc = (R)(a.dst ? (a.inv ? 1.0 / (nx + 1) : 0.5) : (a.inv ? 1.0 / nx : 1.0));
#pragma unroll
    for (int i = 0; i < RPI; ++i) {
      const int row = r0 + g * RPI + i;
      if (row >= a.rows) continue;
      C* orow = out + (size_t)row * a.ld;
#pragma unroll
      for (int k = 0; k < L2; ++k) {
        const int j = k1 + L1 * k;
        if (!a.dst) {
          if (j < nx) orow[j] = mk(acc[i][k].x * sc, acc[i][k].y * sc);
        } else if (j >= 1 && j <= nx) {
          orow[j - 1] = mk(-acc[i][k].y * sc, acc[i][k].x * sc);
        }
      }
    }
  }
}

template <typename C, int L1, int L2, int RPI>
cudaError_t launch_xdft2r(const XfftArgs& a, cudaStream_t st) {
  constexpr int XB = (TT / L2) * RPI;
  const size_t smem = (size_t)(XB + 1) * a.L * sizeof(C) + (size_t)a.L * sizeof(typename TwS<C>::T);
  auto kern = k_xform_dft2r<C, L1, L2, RPI>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<ceil_div(a.rows, XB), TT, smem, st>>>(a);
  return cudaGetLastError();
}

// The same two steps with odd factors fixed at compile time, the FP64 form
// (15 x 17 for the periodic grid of 255 points).  Each length-P DFT (P odd, H = (P-1)/2) folds
// its input into s_n = x_n + x_{P-n} and d_n = x_n - x_{P-n}, n = 1..H, so that
//   X_k     = x_0 + sum_n s_n cos(2 pi n k/P) - i sum_n d_n sin(2 pi n k/P),
//   X_{P-k} = x_0 + sum_n s_n cos(2 pi n k/P) + i sum_n d_n sin(2 pi n k/P)
// (forward root; the inverse swaps the two): H^2 pairs of real-scaled complex
// multiply-adds instead of P^2 complex products.  The loops unroll, every
// table index (n k mod P) is a constant, and each output is emitted as soon as
// it is formed (step 1 back to the positions the item read, step 2 to global
// memory), so a thread holds its P inputs and two accumulators.  (For FP32 this
// form measured slower than the row-pair form above, 0.094 against 0.064 ms
// on the 255 x 255 x 256 workload; for FP64, bound by its FMA rate, it takes
// 0.84 ms against 2.24 ms.)
PD_D float2 cfma_r(float2 acc, float2 x, float r) { return f2fma(x, make_float2(r, r), acc); }
PD_D double2 cfma_r(double2 acc, double2 x, double r) {
  return make_double2(fma(x.x, r, acc.x), fma(x.y, r, acc.y));
}

// cs[q] = (cos, sin)(2 pi q / P), q < P
template <typename C, int P, typename Emit>
PD_D void dft_odd_fold(C* v, const C* cs, bool inv, Emit emit) {
  constexpr int H = (P - 1) / 2;
  C X0 = v[0];
#pragma unroll
  for (int n = 1; n <= H; ++n) {
    const C a = v[n], b = v[P - n];
    v[n] = cadd(a, b);        // s_n
    v[P - n] = csub(a, b);    // d_n
    X0 = cadd(X0, v[n]);
  }
  emit(0, X0);
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    C sc = v[0], ds = czero<C>();
#pragma unroll
    for (int n = 1; n <= H; ++n) {
      const C t = cs[(n * k) % P];
      sc = cfma_r(sc, v[n], t.x);
      ds = cfma_r(ds, v[P - n], t.y);
    }
    const C m = mk(sc.x + ds.y, sc.y - ds.x);   // sc - i ds
    const C q = mk(sc.x - ds.y, sc.y + ds.x);   // sc + i ds
    emit(k, inv ? q : m);
    emit(P - k, inv ? m : q);
  }
}

template <typename C, int L1, int L2>
__global__ void __launch_bounds__(TT) k_xform_dft2f(XfftArgs a) {
  using R = decltype(C::x);
  static_assert((L1 & 1) && (L2 & 1) && L1 <= L2, "odd factors, L1 <= L2");
  constexpr int L = L1 * L2;
  constexpr int XB = TT / L2;            // rows per block
  extern __shared__ __align__(16) unsigned char smraw[];
  C* stp = reinterpret_cast<C*>(smraw);  // [k][n2]: W_L^{n2 k} (conjugated for the inverse)
  C* cs1 = stp + L;                      // (cos, sin)(2 pi q / L1)
  C* cs2 = cs1 + L1;                     // (cos, sin)(2 pi q / L2)
  C* sm = cs2 + L2 + 1;                  // [XB][L] (16-byte aligned: L + L1 + L2 + 1 is even)
  const int nx = a.nx;
  const bool inv = a.inv != 0 && !a.dst;
  const C* tw = reinterpret_cast<const C*>(a.tw);   // W_L^m, m < L (forward root)
  for (int i = threadIdx.x; i < L; i += TT) {
    const int k = i / L2, n2 = i - k * L2;
    C v = tw[n2 * k];
    if (inv) v.y = -v.y;
    stp[i] = v;
  }
  for (int q = threadIdx.x; q < L1 + L2; q += TT) {
    // W_L^{q L2} = cos(2 pi q/L1) - i sin(2 pi q/L1), and likewise for L2
    if (q < L1) {
      const C w = tw[q * L2];
      cs1[q] = mk(w.x, -w.y);
    } else {
      const C w = tw[(q - L1) * L1];
      cs2[q - L1] = mk(w.x, -w.y);
    }
  }
  const int r0 = blockIdx.x * XB;
  const C* in = reinterpret_cast<const C*>(a.in);
  C* out = reinterpret_cast<C*>(a.out);
  for (int e = threadIdx.x; e < XB * L; e += TT) {
    const int r = e / L, m = e - r * L;
    const int row = r0 + r;
    C v = czero<C>();
    if (row < a.rows) {
      if (!a.dst) {
        v = in[(size_t)row * a.ld + m];
      } else if (m >= 1 && m <= nx) {
        v = in[(size_t)row * a.ld + (m - 1)];
      } else if (m >= nx + 2) {
        const C w = in[(size_t)row * a.ld + (L - 1 - m)];
        v = mk(-w.x, -w.y);
      }
    }
    sm[e] = v;
  }
  __syncthreads();
  // step 1: item (row r, n2): the length-L1 DFT over n1, the twiddle W_L^{n2 k1}
  if (threadIdx.x < XB * L2) {
    const int r = threadIdx.x / L2, n2 = threadIdx.x - r * L2;
    C* row = sm + (size_t)r * L;
    C v[L1];
#pragma unroll
    for (int n1 = 0; n1 < L1; ++n1) v[n1] = row[L2 * n1 + n2];
    dft_odd_fold<C, L1>(v, cs1, inv, [&](int k, C X) {
      row[L2 * k + n2] = cmul(X, stp[k * L2 + n2]);
    });
  }
  __syncthreads();
  // step 2: item (row r, k1): the length-L2 DFT over n2, outputs j = k1 + L1 k2
  if (threadIdx.x < XB * L1) {
    const int r = threadIdx.x / L1, k1 = threadIdx.x - r * L1;
    const int row = r0 + r;
    const C* grp = sm + (size_t)r * L + (size_t)L2 * k1;
    C v[L2];
#pragma unroll
    for (int n2 = 0; n2 < L2; ++n2) v[n2] = grp[n2];
    const R sc = (R)(a.dst ? (a.inv ? 1.0 / (nx + 1) : 0.5) : (a.inv ? 1.0 / nx : 1.0));
    C* orow = out + (size_t)(row < a.rows ? row : 0) * a.ld;
    const bool live = row < a.rows;
    dft_odd_fold<C, L2>(v, cs2, inv, [&](int k, C X) {
      const int j = k1 + L1 * k;
      if (!live) return;
      if (!a.dst) {
        if (j < nx) orow[j] = mk(X.x * sc, X.y * sc);
      } else if (j >= 1 && j <= nx) {
        orow[j - 1] = mk(-X.y * sc, X.x * sc);       // (i/2) V_j, scaled
      }
    });
  }
}

template <typename C, int L1, int L2>
cudaError_t launch_xdft2f(const XfftArgs& a, cudaStream_t st) {
  constexpr int XB = TT / L2;
  const size_t smem = ((size_t)XB * a.L + a.L + L1 + L2 + 1) * sizeof(C);
  auto kern = k_xform_dft2f<C, L1, L2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<ceil_div(a.rows, XB), TT, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename C, int B>
cudaError_t launch_xdft2_b(const XfftArgs& a, cudaStream_t st) {
  const int XB = TT / a.L2;
  const size_t smem = ((size_t)XB * a.L + a.L) * sizeof(C);
  auto kern = k_xform_dft2<C, B>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<ceil_div(a.rows, XB), TT, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename C>
cudaError_t launch_xdft2(const XfftArgs& a, cudaStream_t st) {
  // L1 <= L2 <= 32: every item of both steps has a thread (XB L1 <= XB L2 <= 256)
  const int b = a.L2;
  if (a.L1 < 1 || a.L1 > a.L2 || a.L1 * a.L2 != a.L || b > 32) return cudaErrorInvalidValue;
  // the periodic grid of 255 points: factors fixed at compile time
  // the periodic grid of 255 points: factors fixed at compile time; FP32 two
  // rows per item with paired FMAs, FP64 the folded form (fewer FP64 FMAs)
  if (a.L1 == 15 && a.L2 == 17) {
    if constexpr (sizeof(C) == 8) return launch_xdft2r<C, 15, 17, 2>(a, st);
    else return launch_xdft2f<C, 15, 17>(a, st);
  }
  if (b <= 8) return launch_xdft2_b<C, 8>(a, st);
  if (b <= 16) return launch_xdft2_b<C, 16>(a, st);
  if (b <= 24) return launch_xdft2_b<C, 24>(a, st);
  return launch_xdft2_b<C, 32>(a, st);
}

// complex elements per thread needed by a tile of N x TX/2 columns
// complex elements per thread of a tile; the tile budgets of the plans
// (N TX <= 8192 mixed, <= 2048 FP64) keep it at 16 or less
inline int ept_for(int N, int TX) {
  const int e = (N * (TX / 2) + TT - 1) / TT;
  return e <= 4 ? 4 : e <= 8 ? 8 : 16;
}

template <int PREC, int BAND, int EPT>
cudaError_t launch_fwd_e(const FwdArgs& a, cudaStream_t st) {
  const int rows = a.xf.M ? a.xf.M : a.N;
  const size_t smem = (size_t)rows * (a.TX / 2 + 1) * (PREC == 0 ? sizeof(float2) : sizeof(double2));
  auto kern = k_time_fwd<PREC, BAND, EPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = ceil_div(a.S, a.TX);
  kern<<<grid, TT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int PREC, int BAND>
cudaError_t launch_fwd_t(const FwdArgs& a, cudaStream_t st) {
  switch (ept_for(a.xf.M ? a.xf.M : a.N, a.TX)) {
    case 4: return launch_fwd_e<PREC, BAND, 4>(a, st);
    case 8: return launch_fwd_e<PREC, BAND, 8>(a, st);
    default: return launch_fwd_e<PREC, BAND, 16>(a, st);
  }
}

// shared memory of the time kernels: the FFT tile and the twiddle table
inline size_t inv_smem(int N, int rows, int TX, bool fp64, bool upd) {
  (void)N;
  (void)upd;
  return (size_t)rows * (TX / 2 + 1) * (fp64 ? sizeof(double2) : sizeof(float2));
}

template <int PREC, int EPT>
cudaError_t launch_inv_e(const InvArgs& a, cudaStream_t st) {
  const int rows = a.xf.M ? a.xf.M : a.N;
  const bool upd = PREC == 0 ? a.mode == INV_UPDATE_DF : a.mode == INV_UPDATE64;
  const size_t smem = inv_smem(a.N, rows, a.TX, PREC == 1, upd);
  auto kern = k_time_inv<PREC, EPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = ceil_div(a.S, a.TX);
  kern<<<grid, TT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_inv_t(const InvArgs& a, cudaStream_t st) {
  switch (ept_for(a.xf.M ? a.xf.M : a.N, a.TX)) {
    case 4: return launch_inv_e<PREC, 4>(a, st);
    case 8: return launch_inv_e<PREC, 8>(a, st);
    default: return launch_inv_e<PREC, 16>(a, st);
  }
}

// split transforms: a cluster of CR blocks per tile, each with N/CR rows and
// the full element budget (N TX = CR 8192 mixed, CR 2048 FP64)
template <int PREC> constexpr int cl_ept() { return PREC == 0 ? 16 : 4; }

template <int PREC, int BAND, int CR>
cudaError_t launch_fwd_cl(const FwdArgs& a, cudaStream_t st) {
  constexpr int EPT = cl_ept<PREC>();
  const int NL = a.N / CR;
  if (a.xf.M != 0 || NL * CR != a.N || ept_for(NL, a.TX) != EPT) return cudaErrorInvalidValue;
  const size_t smem = (size_t)NL * (a.TX / 2 + 1) * (PREC == 0 ? sizeof(float2) : sizeof(double2));
  // the 1D form only where it changes the code (the mixed residual)
  auto kern = (PREC == 0 && a.st.dim == 1) ? k_time_fwd_cl<PREC, BAND, EPT, CR, true>
                                           : k_time_fwd_cl<PREC, BAND, EPT, CR, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<ceil_div(a.S, a.TX) * CR, TT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int PREC, int CR>
cudaError_t launch_inv_cl(const InvArgs& a, cudaStream_t st) {
  constexpr int EPT = cl_ept<PREC>();
  const int NL = a.N / CR;
  if (a.xf.M != 0 || NL * CR != a.N || ept_for(NL, a.TX) != EPT) return cudaErrorInvalidValue;
  const size_t smem = inv_smem(a.N, NL, a.TX, PREC == 1, true);
  auto kern = k_time_inv_cl<PREC, EPT, CR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<ceil_div(a.S, a.TX) * CR, TT, smem, st>>>(a);
  return cudaGetLastError();
}

template <int PREC, int BAND>
cudaError_t launch_fwd_cl_t(const FwdArgs& a, cudaStream_t st) {
  switch (a.CR) {
    case 2: return launch_fwd_cl<PREC, BAND, 2>(a, st);
    case 4: return launch_fwd_cl<PREC, BAND, 4>(a, st);
    case 8: return launch_fwd_cl<PREC, BAND, 8>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
template <int PREC>
cudaError_t launch_inv_cl_t(const InvArgs& a, cudaStream_t st) {
  switch (a.CR) {
    case 2: return launch_inv_cl<PREC, 2>(a, st);
    case 4: return launch_inv_cl<PREC, 4>(a, st);
    case 8: return launch_inv_cl<PREC, 8>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_time_fwd(const FwdArgs& a, bool fp64, cudaStream_t st) {
  const bool lf = a.tb.band == 2;
  if (a.CR > 1) {
    if (fp64) return lf ? launch_fwd_cl_t<1, 2>(a, st) : launch_fwd_cl_t<1, 1>(a, st);
    return lf ? launch_fwd_cl_t<0, 2>(a, st) : launch_fwd_cl_t<0, 1>(a, st);
  }
  if (fp64) return lf ? launch_fwd_t<1, 2>(a, st) : launch_fwd_t<1, 1>(a, st);
  return lf ? launch_fwd_t<0, 2>(a, st) : launch_fwd_t<0, 1>(a, st);
}

cudaError_t launch_time_inv(const InvArgs& a, bool fp64, cudaStream_t st) {
  if (a.CR > 1) return fp64 ? launch_inv_cl_t<1>(a, st) : launch_inv_cl_t<0>(a, st);
  return fp64 ? launch_inv_t<1>(a, st) : launch_inv_t<0>(a, st);
}

cudaError_t launch_xform_fft(const XfftArgs& a, bool fp64, cudaStream_t st) {
  if (a.rows == 0) return cudaSuccess;
  if (a.L1 > 0) return fp64 ? launch_xdft2<double2>(a, st) : launch_xdft2<float2>(a, st);
  // complex elements per thread of a tile: (M or L) x XR / TT
  const int rows_fft = a.xf.M ? a.xf.M : a.L;
  const int e = (rows_fft * XR + TT - 1) / TT;
  if (fp64) {
    if (e <= 4) return launch_xfft_e<double2, 4>(a, st);
    if (e <= 8) return launch_xfft_e<double2, 8>(a, st);
    if (e <= 16) return launch_xfft_e<double2, 16>(a, st);
  } else {
    if (e <= 4) return launch_xfft_e<float2, 4>(a, st);
    if (e <= 8) return launch_xfft_e<float2, 8>(a, st);
    if (e <= 16) return launch_xfft_e<float2, 16>(a, st);
  }
  return cudaErrorInvalidValue;   // M x XR above 4096 elements: not supported
}

namespace {
template <int PREC, int BAND>
cudaError_t launch_fwd_batch_t(const FwdArgs* descs, const int2* work, int nblocks, size_t smem,
                               int ept, cudaStream_t st) {
#define PD_FWD_B(E)                                                                              \
  {                                                                                              \
    auto kern = k_time_fwd_batch<PREC, BAND, E>;                                                 \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                              \
    kern<<<nblocks, TT, smem, st>>>(descs, work);                                                \
    return cudaGetLastError();                                                                   \
  }
  if (ept <= 4) PD_FWD_B(4)
  if (ept <= 8) PD_FWD_B(8)
  PD_FWD_B(16)
#undef PD_FWD_B
}
template <int PREC>
cudaError_t launch_inv_batch_t(const InvArgs* descs, const int2* work, int nblocks, size_t smem,
                               int ept, cudaStream_t st) {
#define PD_INV_B(E)                                                                              \
  {                                                                                              \
    auto kern = k_time_inv_batch<PREC, E>;                                                       \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                              \
    kern<<<nblocks, TT, smem, st>>>(descs, work);                                                \
    return cudaGetLastError();                                                                   \
  }
  if (ept <= 4) PD_INV_B(4)
  if (ept <= 8) PD_INV_B(8)
  PD_INV_B(16)
#undef PD_INV_B
}
}  // namespace

int time_tile_ept(int N, int TX) { return ept_for(N, TX); }
size_t time_inv_smem(int N, int rows, int TX, bool fp64, bool upd) {
  return inv_smem(N, rows, TX, fp64, upd);
}

cudaError_t launch_time_fwd_batch(const FwdArgs* descs, const int2* work, int nblocks, int band,
                                  size_t smem, int ept, bool fp64, cudaStream_t st) {
  if (nblocks == 0) return cudaSuccess;
  if (fp64) return band == 2 ? launch_fwd_batch_t<1, 2>(descs, work, nblocks, smem, ept, st)
                             : launch_fwd_batch_t<1, 1>(descs, work, nblocks, smem, ept, st);
  return band == 2 ? launch_fwd_batch_t<0, 2>(descs, work, nblocks, smem, ept, st)
                   : launch_fwd_batch_t<0, 1>(descs, work, nblocks, smem, ept, st);
}

cudaError_t launch_time_inv_batch(const InvArgs* descs, const int2* work, int nblocks,
                                  size_t smem, int ept, bool fp64, cudaStream_t st) {
  if (nblocks == 0) return cudaSuccess;
  return fp64 ? launch_inv_batch_t<1>(descs, work, nblocks, smem, ept, st)
              : launch_inv_batch_t<0>(descs, work, nblocks, smem, ept, st);
}
