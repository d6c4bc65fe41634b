// Step (b) of eq. 1.3: the Nt independent complex-shifted spatial solves
// (lambda_1 I + lambda_2 K) z = s, here for the constant-coefficient
// tridiagonal K of one direction (1D problems, or y after the x-eigentransform
// of 2D problems, where the shift also carries the x-eigenvalue mu_j).
//
// Partitioned solver, no pivoting.  L lanes cooperate on one system of length
// n; lane G owns the m = ceil(n / L) consecutive rows i0 = G m .. i0 + m - 1
// (the last lanes own fewer, possibly none).  Rows are scaled by 1/d so the
// diagonal is one: l z_{i-1} + z_i + u z_{i+1} = s_i / d.
//
// Every system is Toeplitz, so the elimination of the interior rows
// t = 1 .. m-2 of a chunk, in terms of the chunk's first unknown f and last
// unknown g, uses the same factors in every chunk:
//   forward   yh_t = s_t a_t - b_t yh_{t-1},   a_t = iden_t / d, b_t = l iden_t,
//             iden_t = 1 / (1 - l cc_{t-1}),   cc_t = u iden_t,
//             ph_t = -b_t ph_{t-1} (ph_0 = 1)  (the dependence on f),
//   backward  z_t = yh_t + ph_t f - cc_t z_{t+1},  z_{mi+1} = g.
// Unrolling the backward sweep, z_1 = sum_t w_t yh_t + P_1 f + Q_1 g with
// w_t = prod_{s<t} (-cc_s), P_1 = sum_{t<=mi} w_t ph_t and Q_1 = w_{mi+1}.
// One thread per system builds the table (a, b, ph, cc, w) in shared memory;
// the L lanes of the system then run one forward sweep over their registers,
// form the two reduced rows of the chunk (f at 2G, g at 2G+1), solve the
// reduced tridiagonal system of 2L unknowns by parallel cyclic reduction
// (warp shuffles for L <= 32, shared memory otherwise), and finish with the
// backward sweep.  A chunk that ends at row n-1 early (the boundary lane) is
// the leading part of a full chunk, so it uses the same table and only its own
// P_1, Q_1.
#include <algorithm>
#include <cstring>

#include "pd_internal.h"

namespace {

// rows per chunk held in registers (compile-time bound of the unrolled sweeps):
// 32 (FP32) or 16 (FP64) by default; FP32 plans may also take the 16-row form
// (half the registers, twice the lanes per system), which the plan-time
// autotuner weighs against the default
template <typename R> struct ChunkRows;
template <> struct ChunkRows<float> { static constexpr int MM = 32; };
template <> struct ChunkRows<double> { static constexpr int MM = 16; };

// threads per block and systems per block for L lanes per system
__host__ __device__ constexpr int tri_threads(int L) { return L >= 128 ? L : (16 * L < 32 ? 32 : (16 * L > 128 ? 128 : 16 * L)); }
__host__ __device__ constexpr int tri_sb(int L) { return tri_threads(L) / L; }

template <typename C>
struct Row4 { C a, b, c, d; };

// complex reciprocal; in FP32 with the hardware reciprocal (rcp.approx, a few
// ulp), which is ample for a preconditioner whose residual is formed apart
PD_D float2 trcp(float2 a) {
  float s;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(fmaf(a.x, a.x, a.y * a.y)));
  return make_float2(a.x * s, -a.y * s);
}
PD_D double2 trcp(double2 a) { return crcp(a); }

// one entry of the per-system elimination table (interior row t)
template <typename C>
struct alignas(16) TabRow { C a, b, ph, cc, w, pad; };

template <typename C>
struct SysInfo {
  C ld, ud, invd;
  C P1, Q1;      // full chunks
  C P1b, Q1b;    // the boundary chunk (rows up to n-1)
  long long base;
};

template <int L, typename C>
PD_D C shfl_up_c(C v, int d) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, d, L);
  v.y = __shfl_up_sync(0xffffffffu, v.y, d, L);
  return v;
}
template <int L, typename C>
PD_D C shfl_down_c(C v, int d) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, d, L);
  v.y = __shfl_down_sync(0xffffffffu, v.y, d, L);
  return v;
}
template <int L, typename C>
PD_D Row4<C> shfl_up_r(const Row4<C>& r, int d) {
  Row4<C> o;
  o.a = shfl_up_c<L>(r.a, d); o.b = shfl_up_c<L>(r.b, d);
  o.c = shfl_up_c<L>(r.c, d); o.d = shfl_up_c<L>(r.d, d);
  return o;
}
template <int L, typename C>
PD_D Row4<C> shfl_down_r(const Row4<C>& r, int d) {
  Row4<C> o;
  o.a = shfl_down_c<L>(r.a, d); o.b = shfl_down_c<L>(r.b, d);
  o.c = shfl_down_c<L>(r.c, d); o.d = shfl_down_c<L>(r.d, d);
  return o;
}

// one PCR elimination of row x with its neighbours at distance s (absent
// neighbours lie outside the system and contribute nothing)
template <typename C>
PD_D Row4<C> pcr_step(const Row4<C>& x, const Row4<C>& m, bool hm, const Row4<C>& p, bool hp) {
  Row4<C> o;
  o.a = czero<C>(); o.c = czero<C>(); o.b = x.b; o.d = x.d;
  if (hm) {
    const C k1 = cmul(x.a, trcp(m.b));
    o.a = mk(-(m.a.x * k1.x - m.a.y * k1.y), -(m.a.x * k1.y + m.a.y * k1.x));
    o.b = csub(o.b, cmul(m.c, k1));
    o.d = csub(o.d, cmul(m.d, k1));
  }
  if (hp) {
    const C k2 = cmul(x.c, trcp(p.b));
    o.c = mk(-(p.c.x * k2.x - p.c.y * k2.y), -(p.c.x * k2.y + p.c.y * k2.x));
    o.b = csub(o.b, cmul(p.a, k2));
    o.d = csub(o.d, cmul(p.d, k2));
  }
  return o;
}

template <typename C>
PD_D Row4<C> ident_row() {
  Row4<C> r;
  r.a = czero<C>(); r.c = czero<C>(); r.d = czero<C>();
  r.b = czero<C>(); r.b.x = 1;
  return r;
}

// Table of one system (one thread): coefficients, the interior factors of a
// chunk of m rows and the P_1, Q_1 of full and boundary chunks.
template <typename R>
PD_D void build_table(const TriArgs& a, long long q, int m, TabRow<cplx_t<R>>* tab,
                      SysInfo<cplx_t<R>>* info) {
  using C = cplx_t<R>;
  const long long k = q / a.J, j = q % a.J;
  const C* lam = reinterpret_cast<const C*>(a.lam);
  const C l1 = lam[2 * k], l2 = lam[2 * k + 1];
  C mu = czero<C>();
  if (a.mu != nullptr) mu = reinterpret_cast<const C*>(a.mu)[j];
  const C d = cadd(l1, cmul(l2, cadd(mk((R)a.cd, (R)0), mu)));
  const C invd = trcp(d);
  const C ld = cmul(cscale(l2, (R)a.cl), invd);
  const C ud = cmul(cscale(l2, (R)a.cu), invd);
  const int n = a.n;
  const int mi = m - 2;
  const int mob = n - ((n - 1) / m) * m;  // rows of the boundary chunk (1 .. m)
  const int mib = mob - 2;
  const C one = mk((R)1, (R)0);
  C cc = czero<C>(), ph = one, w = one, pp = czero<C>();
  C P1 = czero<C>(), Q1 = czero<C>(), P1b = czero<C>(), Q1b = czero<C>();
  for (int t = 1; t <= mi; ++t) {
    const C iden = trcp(csub(one, cmul(ld, cc)));
    TabRow<C> e;
    e.a = cmul(iden, invd);
    e.b = cmul(ld, iden);
    cc = cmul(ud, iden);
    ph = cmul(e.b, ph);
    ph.x = -ph.x; ph.y = -ph.y;
    pp = cadd(pp, cmul(w, ph));
    e.ph = ph;
    e.cc = cc;
    e.w = w;
    e.pad = czero<C>();
    tab[t - 1] = e;
    w = cmul(w, cc);
    w.x = -w.x; w.y = -w.y;  // w_{t+1}
    if (t == mi) { P1 = pp; Q1 = w; }
    if (t == mib) { P1b = pp; Q1b = w; }
  }
  info->ld = ld; info->ud = ud; info->invd = invd;
  info->P1 = P1; info->Q1 = Q1; info->P1b = P1b; info->Q1b = Q1b;
  info->base = k * a.S + j;
}

template <typename C>
PD_D void ld_pair(const C* p, C& x, C& y);
template <>
PD_D void ld_pair<float2>(const float2* p, float2& x, float2& y) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x = make_float2(v.x, v.y);
  y = make_float2(v.z, v.w);
}
template <>
PD_D void ld_pair<double2>(const double2* p, double2& x, double2& y) {
  x = p[0];
  y = p[1];
}

// Solve the SB systems of one tile: q0 + sb for sb < SB.  Block threads:
// sb = threadIdx.x / L, lane G = threadIdx.x % L.
template <typename R, int L, int MM>
PD_D void solve_tile(const TriArgs& a, long long q0, unsigned char* smraw) {
  using C = cplx_t<R>;
  constexpr int SB = tri_sb(L);
  TabRow<C>* tab = reinterpret_cast<TabRow<C>*>(smraw);                   // [SB][MM-2]
  SysInfo<C>* sinfo = reinterpret_cast<SysInfo<C>*>(tab + SB * (MM - 2));  // [SB]
  C* pcr = reinterpret_cast<C*>(sinfo + SB);                                // [4][SB][2L] (L > 32)

  const int n = a.n;
  const int m = max(2, (n + L - 1) / L);
  const long long total = (long long)a.nh * a.J;
  const int sb = threadIdx.x / L, G = threadIdx.x % L;
  const long long q = q0 + sb;
  const bool active = q < total;
  const int i0 = G * m;
  const int mown = active ? max(0, min(m, n - i0)) : 0;
  C* data = reinterpret_cast<C*>(a.data);

  // right-hand side of this chunk into registers (all loads in flight while
  // the tables are built)
  C sv[MM];
  long long base = 0;
  if (active) {
    const long long k = q / a.J, j = q % a.J;
    base = k * a.S + j;
  }
  const C* src = data + base + (long long)i0 * a.stride;
#pragma unroll
  for (int t = 0; t < MM; ++t)
    sv[t] = (t < mown) ? src[(long long)t * a.stride] : czero<C>();
  C slast = czero<C>();
  if (mown >= 2) slast = src[(long long)(mown - 1) * a.stride];

  for (int s = threadIdx.x; s < SB; s += blockDim.x)
    if (q0 + s < total) build_table<R>(a, q0 + s, m, tab + s * (MM - 2), sinfo + s);
  __syncthreads();

  const TabRow<C>* tb = tab + sb * (MM - 2);
  C ld = czero<C>(), ud = czero<C>(), invd = czero<C>(), P1x = czero<C>(), Q1x = czero<C>();
  if (active) {
    const SysInfo<C>& si = sinfo[sb];
    ld = si.ld; ud = si.ud; invd = si.invd;
    P1x = (mown == m) ? si.P1 : si.P1b;
    Q1x = (mown == m) ? si.Q1 : si.Q1b;
  }
  const int mi = mown - 2;

  // ---- forward sweep over the interior rows (yh overwrites s)
  C y = czero<C>(), Y1 = czero<C>();
#pragma unroll
  for (int t = 1; t < MM - 1; ++t) {
    if (t > mi) break;
    C at, bt;
    ld_pair(&tb[t - 1].a, at, bt);
    const C wt = tb[t - 1].w;
    const C s = sv[t];
    y = mk(s.x * at.x - s.y * at.y - (bt.x * y.x - bt.y * y.y),
           s.x * at.y + s.y * at.x - (bt.x * y.y + bt.y * y.x));
    sv[t] = y;
    Y1 = cadd(Y1, cmul(wt, y));
  }

  // ---- reduced rows
  const C one = mk((R)1, (R)0);
  Row4<C> rf = ident_row<C>(), rg = ident_row<C>();
  if (mown >= 1) {
    const C s0 = cmul(sv[0], invd);
    const C l0 = G > 0 ? ld : czero<C>();
    if (mown == 1) {
      rf.a = l0; rf.b = one; rf.c = czero<C>(); rf.d = s0;
    } else {
      const C sl = cmul(slast, invd);
      const C ul = (i0 + mown < n) ? ud : czero<C>();
      if (mi >= 1) {
        C phm, ccm;
        ld_pair(&tb[mi - 1].ph, phm, ccm);
        rf.a = l0;
        rf.b = cadd(one, cmul(ud, P1x));
        rf.c = cmul(ud, Q1x);
        rf.d = csub(s0, cmul(ud, Y1));
        rg.a = cmul(ld, phm);
        rg.b = csub(one, cmul(ld, ccm));
        rg.c = ul;
        rg.d = csub(sl, cmul(ld, y));
      } else {
        rf.a = l0; rf.b = one; rf.c = ud; rf.d = s0;
        rg.a = ld; rg.b = one; rg.c = ul; rg.d = sl;
      }
    }
  }

  // ---- PCR on the reduced system of 2L rows
  C f, g;
  if constexpr (L <= 32) {
    for (int s = 1; s < 2 * L; s <<= 1) {
      Row4<C> mf, pf, mg, pg;
      bool hmf, hpf, hmg, hpg;
      if (s == 1) {
        const Row4<C> gm = shfl_up_r<L>(rg, 1);    // row 2G-1
        const Row4<C> fp = shfl_down_r<L>(rf, 1);  // row 2G+2
        mf = gm; hmf = G > 0;  pf = rg; hpf = true;
        mg = rf; hmg = true;   pg = fp; hpg = G < L - 1;
      } else {
        const int d = s >> 1;
        mf = shfl_up_r<L>(rf, d); mg = shfl_up_r<L>(rg, d);
        pf = shfl_down_r<L>(rf, d); pg = shfl_down_r<L>(rg, d);
        hmf = hmg = G >= d;
        hpf = hpg = G + d < L;
      }
      const Row4<C> nf = pcr_step(rf, mf, hmf, pf, hpf);
      const Row4<C> ng = pcr_step(rg, mg, hmg, pg, hpg);
      rf = nf;
      rg = ng;
    }
    f = cmul(rf.d, trcp(rf.b));
    g = cmul(rg.d, trcp(rg.b));
  } else {
    constexpr int R2 = 2 * L;
    C* A_ = pcr + (size_t)sb * R2;
    C* B_ = A_ + (size_t)SB * R2;
    C* C_ = B_ + (size_t)SB * R2;
    C* D_ = C_ + (size_t)SB * R2;
    const int rf_i = 2 * G, rg_i = 2 * G + 1;
    A_[rf_i] = rf.a; B_[rf_i] = rf.b; C_[rf_i] = rf.c; D_[rf_i] = rf.d;
    A_[rg_i] = rg.a; B_[rg_i] = rg.b; C_[rg_i] = rg.c; D_[rg_i] = rg.d;
    __syncthreads();
    for (int s = 1; s < R2; s <<= 1) {
      Row4<C> nw[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = 2 * G + h;
        const int im = i - s, ip = i + s;
        Row4<C> x, mr, pr;
        x.a = A_[i]; x.b = B_[i]; x.c = C_[i]; x.d = D_[i];
        mr = x; pr = x;
        if (im >= 0) { mr.a = A_[im]; mr.b = B_[im]; mr.c = C_[im]; mr.d = D_[im]; }
        if (ip < R2) { pr.a = A_[ip]; pr.b = B_[ip]; pr.c = C_[ip]; pr.d = D_[ip]; }
        nw[h] = pcr_step(x, mr, im >= 0, pr, ip < R2);
      }
      __syncthreads();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = 2 * G + h;
        A_[i] = nw[h].a; B_[i] = nw[h].b; C_[i] = nw[h].c; D_[i] = nw[h].d;
      }
      __syncthreads();
    }
    f = cmul(D_[rf_i], trcp(B_[rf_i]));
    g = cmul(D_[rg_i], trcp(B_[rg_i]));
  }

  // ---- backward sweep and store
  bool bad = false;
  C* dst = data + base + (long long)i0 * a.stride;
  C z = g;
#pragma unroll
  for (int t = MM - 2; t >= 1; --t) {
    if (t <= mi) {
      C ph, cc;
      ld_pair(&tb[t - 1].ph, ph, cc);
      const C yh = sv[t];
      z = mk(yh.x + ph.x * f.x - ph.y * f.y - (cc.x * z.x - cc.y * z.y),
             yh.y + ph.x * f.y + ph.y * f.x - (cc.x * z.y + cc.y * z.x));
      sv[t] = z;
    }
  }
#pragma unroll
  for (int t = 1; t < MM - 1; ++t) {
    if (t <= mi) {
      const C v = sv[t];
      bad |= !(isfinite(v.x) && isfinite(v.y));
      dst[(long long)t * a.stride] = v;
    }
  }
  if (mown >= 1) {
    bad |= !(isfinite(f.x) && isfinite(f.y));
    dst[0] = f;
  }
  if (mown >= 2) {
    bad |= !(isfinite(g.x) && isfinite(g.y));
    dst[(long long)(mown - 1) * a.stride] = g;
  }
  if (bad && a.flag != nullptr) atomicOr(a.flag, 1);
  if constexpr (sizeof(R) == 4) {
    // largest |solution| for the scaling of the tensor-core x-transform
    if (a.amax != nullptr) {
      float mx = 0.f;
      if (mown >= 1) mx = fmaxf(fabsf(f.x), fabsf(f.y));
      if (mown >= 2) mx = fmaxf(mx, fmaxf(fabsf(g.x), fabsf(g.y)));
#pragma unroll
      for (int t = 1; t < MM - 1; ++t)
        if (t <= mi) mx = fmaxf(mx, fmaxf(fabsf(sv[t].x), fabsf(sv[t].y)));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if ((threadIdx.x & 31) == 0) atomicMax(a.amax, __float_as_uint(mx));
      if (a.amax_reset != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *a.amax_reset = 0u;
    }
  }
}

// One tile of SB systems per block.  Batch: work[block] = (problem, tile)
// selects the descriptor.
template <typename R, int L, bool BATCH, int MM>
__global__ void __launch_bounds__(tri_threads(L),
                                  L >= 64 ? 1 : (sizeof(R) == 4 ? (MM <= 16 ? 5 : 4) : 2))
    k_tridiag(TriArgs a1, const TriArgs* __restrict__ descs, const int2* __restrict__ work,
              int nwork, int* counter) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (!BATCH) {
    solve_tile<R, L, MM>(a1, (long long)blockIdx.x * tri_sb(L), smraw);
    return;
  }
  // batch: persistent, every block takes the next tile from the device
  // counter (zeroed before the launch) until the table is exhausted
  __shared__ int slot;
  for (;;) {
    __syncthreads();                            // the previous tile is done (shared memory, slot)
    if (threadIdx.x == 0) slot = atomicAdd(counter, 1);
    __syncthreads();
    const int i = slot;
    if (i >= nwork) break;
    const int2 w = work[i];
    solve_tile<R, L, MM>(descs[w.x], (long long)w.y * tri_sb(L), smraw);
  }
}

template <typename R, int L, int MM>
size_t tile_smem() {
  using C = cplx_t<R>;
  constexpr int SB = tri_sb(L);
  size_t b = (size_t)SB * (MM - 2) * sizeof(TabRow<C>) + (size_t)SB * sizeof(SysInfo<C>);
  if (L > 32) b += (size_t)4 * SB * 2 * L * sizeof(C);
  return b;
}

template <typename R, int L, int MM>
cudaError_t launch_l(const TriArgs& a1, const TriArgs* descs, const int2* work, long long ntiles,
                     int* counter, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  const size_t smem = tile_smem<R, L, MM>();
  auto kern = descs ? k_tridiag<R, L, true, MM> : k_tridiag<R, L, false, MM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  long long grid = ntiles;
  if (descs) {
    // persistent batch launch: the resident blocks of the whole GPU
    static int nsm = 0;
    if (nsm == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (nsm <= 0) nsm = 1;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tri_threads(L), smem) !=
            cudaSuccess || per_sm < 1)
      per_sm = 1;
    grid = std::min<long long>(ntiles, (long long)per_sm * nsm);
  }
  kern<<<(unsigned)grid, tri_threads(L), smem, st>>>(a1, descs, work, (int)ntiles, counter);
  return cudaGetLastError();
}

template <typename R, int MM = ChunkRows<R>::MM>
cudaError_t launch_cls(int cls, const TriArgs& a1, const TriArgs* descs, const int2* work,
                       long long ntiles, cudaStream_t st, int* counter = nullptr) {
  switch (cls) {
    case 0: return launch_l<R, 1, MM>(a1, descs, work, ntiles, counter, st);
    case 1: return launch_l<R, 2, MM>(a1, descs, work, ntiles, counter, st);
    case 2: return launch_l<R, 4, MM>(a1, descs, work, ntiles, counter, st);
    case 3: return launch_l<R, 8, MM>(a1, descs, work, ntiles, counter, st);
    case 4: return launch_l<R, 16, MM>(a1, descs, work, ntiles, counter, st);
    case 5: return launch_l<R, 32, MM>(a1, descs, work, ntiles, counter, st);
    case 6: return launch_l<R, 64, MM>(a1, descs, work, ntiles, counter, st);
    case 7: return launch_l<R, 128, MM>(a1, descs, work, ntiles, counter, st);
    case 8: return launch_l<R, 256, MM>(a1, descs, work, ntiles, counter, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int tridiag_class(int n, bool fp64, int rows) {
  const int mm = rows > 0 ? rows : (fp64 ? ChunkRows<double>::MM : ChunkRows<float>::MM);
  if (n < 1 || n > TRI_NMAX) return -1;
  int cls = 0;
  while ((1 << cls) * mm < n) ++cls;
  return cls < TRI_NCLASS ? cls : -1;
}

int tridiag_batch_sb(int cls, bool fp64) {
  (void)fp64;
  return tri_sb(1 << cls);
}

cudaError_t launch_tridiag(const TriArgs& a, bool fp64, cudaStream_t st) {
  const bool short_rows = !fp64 && a.rows == 16;       // the 16-row FP32 form
  const int c0 = tridiag_class(a.n, fp64, short_rows ? 16 : 0);
  if (c0 < 0) return cudaErrorInvalidValue;
  const int cls = a.cls > c0 && a.cls < TRI_NCLASS ? a.cls : c0;
  const long long total = (long long)a.nh * a.J;
  const long long ntiles = (total + tri_sb(1 << cls) - 1) / tri_sb(1 << cls);
  if (fp64) return launch_cls<double>(cls, a, nullptr, nullptr, ntiles, st);
  if (short_rows) return launch_cls<float, 16>(cls, a, nullptr, nullptr, ntiles, st);
  return launch_cls<float>(cls, a, nullptr, nullptr, ntiles, st);
}

cudaError_t launch_tridiag_batch(const TriArgs* descs, const int2* work, int ntiles, int cls,
                                 bool fp64, int* counter, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  TriArgs dummy;
  memset(&dummy, 0, sizeof(dummy));
  return fp64 ? launch_cls<double>(cls, dummy, descs, work, ntiles, st, counter)
              : launch_cls<float>(cls, dummy, descs, work, ntiles, st, counter);
}
