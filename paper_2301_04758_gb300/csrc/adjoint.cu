// Adjoint sweep and cross-section gradients (not in the paper; follows from its transport
// equation).  For R = sum g . phi with phi = sum_d w_d psi_d and L_d psi_d = b_d, the adjoint
// directions solve L_d^T lambda_d = w_d g.  Writing L_d = blockdiag(A_e) + C with the
// upwind coupling blocks C[e'][e] (receiver e', donor e), block row e of L^T reads
//     A_e^T lambda_e = w_d g_e - sum_{e' receiving from e} C[e'][e]^T lambda_{e'}.
// With r_e := A_e^T lambda_e and the stored W_{e',f'} = A_{e'}^{-1} Cin_{e',f'} of the
// forward factorisation, C[e'][e]^T lambda_{e'} = W_{e',f'}^T r_{e'} placed on e's face
// nodes, so each element needs its downstream neighbours' r, and lambda_e = A_e^{-T} r_e.
// The sweep therefore runs the forward schedule backwards (downwind order): one CTA per
// direction with the forward sweep's shared-memory slots (the default), or one
// thread-block cluster per direction.
//   dR/dsigma_t,e = - sum_d lambda_{d,e}^T M_e psi_{d,e}
//   dR/dsigma_s,e =   sum_d lambda_{d,e}^T M_e phi_in,e / (4 pi)
#include <algorithm>
#include <cmath>

#include "device.cuh"

namespace vef {

constexpr uint32_t kAdjWaitIters = 1u << 18;   // bounded staging waits (~1 s, as the forward sweep's)

struct AdjArgs {
  const int* dir_lev0;
  const int* lev_begin;
  const int* lev_gbegin;
  const int* lev_mbegin;
  const uint4* tslot;     // single-CTA sweep: the forward schedule's slot ids (roles swapped)
  const double* yadj;     // single-CTA sweep: w_d g_e rows per member (16-byte padded)
  int ring;               // single-CTA sweep: chunk buffers in the ring
  int tr_bytes;           // single-CTA sweep: bytes of the trace slots
  const uint32_t* member_nbpos;  // coupled groups solved directly: in-group neighbour positions
  const int* slot_gid;           //   per slot its group index or -1 (null: none solved directly)
  const long long* grp_toff;     //   offset of each group's trace-system inverse in grec
  const double* grec;            //   T = (I + R)^{-1} per group, column-major (forward factorisation)
  int cluster_size;
  const int* slot_first;
  const int* slot_count;
  const uint32_t* code;
  const int* member_of;
  const uint16_t* finfo;
  const double* omega;
  const double* weights;
  const double* rec;      // staged record array S (see Rec)
  const double* recx;     // extra record array X
  long long nmem;
  const double* g;        // [E][n]
  const double* psi;      // [D][E][n] forward checkpoint (FP64), or
  const float* psi32;     //   its FP32 copy (VEF_CKPT_FP32)
  const double* Mm;       // [E][n][n]
  const double* mphi;     // [E][n] M phi_in or null
  const uint32_t* link;   // [members][4] receiver member and W slot across each face
  double* radj;           // [D][E][n] adjoint right-hand sides r
  double* lambda;         // [D][E][n]
  double* dst;            // [E]
  double* dss;            // [E]
  unsigned int* status;
  int nx, ny;
  long long E;
  double tol;
  int max_inner;
};

// r_i of element e (lane = dof row i): w_d g_i minus the downstream couplings on e's faces
// (CG: the receivers' r are read at L2, as a cluster's other CTAs wrote them; in the
// single-CTA sweep this SM wrote them, and they are read with ordinary loads)
template <int P, bool CG = true>
__device__ __forceinline__ double adj_rhs(const AdjArgs& a, int d, int e, long long m, int i, uint16_t bits,
                                          int first, int pos_self, int cnt, int it, bool in_group) {
  constexpr int Q = P + 1, N = Q * Q;
  using L = Rec<P, double>;
  double r = a.weights[d] * a.g[(size_t)e * N + i];
  const int ia = i % Q, ib = i / Q;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (!(bits & (1u << (8 + f)))) continue;   // no receiver across f
    int t = -1;
    if (f == 0 && ib == 0) t = ia;
    if (f == 1 && ia == P) t = ib;
    if (f == 2 && ib == P) t = ia;
    if (f == 3 && ia == 0) t = ib;
    if (t < 0) continue;
    const int nb = nb_elem(a.nx, a.ny, e, f);
    if (in_group && (bits & (1u << (4 + f))) && it == 0) {
      const int pos = a.member_of[(size_t)d * a.E + nb] - first;
      if (pos <= pos_self) continue;  // processed later in the first backward pass
    }
    const uint32_t lk = a.link[m * 4 + f];   // receiver and its W slot for the face toward e
    if (lk == ~0u) continue;
    const long long mn = (long long)(lk >> 2);
    const double* W = L::slot(L::s_at(a.rec, mn), L::x_at(a.recx, mn), (int)(lk & 3u)) + t * N;
    const double* rn = a.radj + ((size_t)d * a.E + nb) * N;
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) s += W[j] * (CG ? __ldcg(rn + j) : rn[j]);
    r -= s;
  }
  (void)cnt;
  return r;
}

template <int P>
__device__ __forceinline__ void adj_finish(const AdjArgs& a, long long m, int d, int e, int i, bool act,
                                           double r) {
  // lambda = A^{-T} r, gradient contributions
  constexpr int Q = P + 1, N = Q * Q;
  using L = Rec<P, double>;
  (void)Q;
  const int lane = threadIdx.x & 31;
  const int base = (lane / N) * N;
  const double* Ai = L::ainv(L::x_at(a.recx, m)) + (size_t)i * N;  // column i of A^{-1}
  double lam = 0.0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const double rj = __shfl_sync(0xffffffffu, r, (base + j) & 31);
    if (act) lam += Ai[j] * rj;
  }
  double gt = 0.0, gs = 0.0;
  if (act) {
    a.lambda[((size_t)d * a.E + e) * N + i] = lam;
    const double* Mr = a.Mm + ((size_t)e * N + i) * N;
    const size_t o = ((size_t)d * a.E + e) * N;
    double mp = 0.0;
    if (a.psi32) {
#pragma unroll
      for (int j = 0; j < N; ++j) mp += Mr[j] * (double)a.psi32[o + j];
    } else {
#pragma unroll
      for (int j = 0; j < N; ++j) mp += Mr[j] * a.psi[o + j];
    }
    gt = -lam * mp;
    if (a.mphi) gs = lam * a.mphi[(size_t)e * N + i] / kFourPi;
  }
  // reduce over the N lanes of the task
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ot = __shfl_down_sync(0xffffffffu, gt, off);
    const double os = __shfl_down_sync(0xffffffffu, gs, off);
    const int src = lane + off;
    if (src < 32 && (src / N) == (lane / N)) { gt += ot; gs += os; }
  }
  if (act && i == 0) {
    atomicAdd(a.dst + e, gt);
    if (a.mphi) atomicAdd(a.dss + e, gs);
  }
}

// One thread-block cluster per direction walks the direction's levels backwards; the
// receivers of a task sit at later levels, so they are complete after the previous
// cluster barrier.
template <int P, bool CG = true>
__device__ __forceinline__ void adj_group(const AdjArgs& a, int d, int s0) {
  constexpr int Q = P + 1, N = Q * Q;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int first = a.slot_first[s0];
  const int cnt = a.slot_count[s0];
  const int i = lane;
  const bool act = lane < N;
  int it = 0;
  bool conv = false;
  for (; it < a.max_inner; ++it) {
    double dmax = 0, amax = 0;
    for (int mi = cnt - 1; mi >= 0; --mi) {
      const int e = (int)(a.code[first + mi] & 0x3fffffu);
      const uint16_t bits = a.finfo[(size_t)d * a.E + e];
      if (act) {
        const double r = adj_rhs<P, CG>(a, d, e, first + mi, i, bits, first, mi, cnt, it, true);
        double* o = a.radj + ((size_t)d * a.E + e) * N + i;
        if (it > 0) dmax = fmax(dmax, fabs(r - (CG ? __ldcg(o) : *o)));
        amax = fmax(amax, fabs(r));
        *o = r;
      }
      __syncwarp();
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(FULL, dmax, off));
      amax = fmax(amax, __shfl_xor_sync(FULL, amax, off));
    }
    if (it > 0 && dmax <= a.tol * amax) { conv = true; ++it; break; }
  }
  if (lane == 0) {
    if (!conv) atomicOr(a.status, kDevNotConverged);
    atomicMax(a.status + 2, (unsigned)it);
  }
}

template <int P>
__global__ void __maxnreg__(128) adjoint_kernel(AdjArgs a) {
  constexpr int Q = P + 1, N = Q * Q;
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  (void)Q;
  const int lane = threadIdx.x & 31;
  const int cs = a.cluster_size;
  const int d = blockIdx.x / cs;
  const int nw = cs * (blockDim.x >> 5);
  const int gw = (blockIdx.x % cs) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int k0 = a.dir_lev0[d], k1 = a.dir_lev0[d + 1];
  const int i = lane % N;
  for (int k = k1 - 1; k >= k0; --k) {
    const int sb = a.lev_begin[k], sg = a.lev_gbegin[k], se = a.lev_begin[k + 1];
    for (int base = sb + gw * SPC; base < sg; base += nw * SPC) {
      const int slot = base + lane / N;
      const bool valid = (lane < SPC * N) && (slot < sg);
      long long m = 0;
      int e = 0;
      double r = 0.0;
      if (valid) {
        m = a.slot_first[slot];
        e = (int)(a.code[m] & 0x3fffffu);
        const uint16_t bits = a.finfo[(size_t)d * a.E + e];
        r = adj_rhs<P>(a, d, e, m, i, bits, 0, 0, 1, 1, false);
        a.radj[((size_t)d * a.E + e) * N + i] = r;
      }
    }
    for (int gs = sg + gw; gs < se; gs += nw) adj_group<P>(a, d, gs);
    cluster_barrier();
  }
}

// Coupled group solved directly in the backward sweep.  The forward group operator is
// L_G = A (I + W P) (W = A^{-1} Cin of the internal faces, P takes the neighbours'
// face-node values), with L_G^{-1} = (I - W T P) A^{-1} and T = (I + P W)^{-1} formed by
// the forward factorisation.  For the adjoint, r = A^T lambda solves
//     r = (I - P^T T^T W^T) g~,   g~ = w_d g - (couplings from receivers outside the group),
// i.e. v = W^T g~ (one value per trace unknown), w = T^T v, r = g~ - P^T w.
template <int P>
struct AdjGroupSmem {
  static constexpr int Q = P + 1, N = Q * Q, GM = group_direct_members(P);
  static constexpr int NC = kGroupMaxTrace / Q + 1;
  double z[GM * N];                                 // g~, then r
  double v[kGroupMaxTrace];
  double w[kGroupMaxTrace];
  double tinv[kGroupSmemTrace * kGroupSmemTrace];   // T (column-major) when nt <= kGroupSmemTrace
  uint4 info[GM];
  uint32_t cpl[NC];                                 // coupling: a | f << 8 | b << 16 | W slot << 24
  int cbase[GM + 1];
  int m, nt, gid;
};

template <int P>
__device__ __forceinline__ void adj_group_stage(const AdjArgs& a, int s0, AdjGroupSmem<P>& g) {
  constexpr int Q = P + 1;
  using L = Rec<P, double>;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int first = a.slot_first[s0];
  const int cnt = a.slot_count[s0];
  const int gid = a.slot_gid[s0];
  uint4 info = make_uint4(0u, 0u, 0xffffffffu, 0u);
  uint32_t nbp = 0xffffffffu;
  if (lane < cnt) {
    info = *reinterpret_cast<const uint4*>(L::s_at(a.rec, first + lane));
    nbp = a.member_nbpos[first + lane];
    g.info[lane] = info;
  }
  const unsigned mine = lane < cnt ? (unsigned)__popc(info.y & (info.y >> 4) & 0xfu) : 0u;
  unsigned incl = mine;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned v = __shfl_up_sync(FULL, incl, off);
    if (lane >= off) incl += v;
  }
  unsigned c = incl - mine;
  if (lane < cnt) {
    g.cbase[lane] = (int)c;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!((info.y >> f) & 1u) || !((info.y >> (4 + f)) & 1u)) continue;
      g.cpl[c++] = (uint32_t)lane | ((uint32_t)f << 8) | (((nbp >> (8 * f)) & 0xffu) << 16) |
                   ((uint32_t)rec_slot_of(info.z, f) << 24);
    }
  }
  const int total = (int)__shfl_sync(FULL, incl, 31);
  if (lane == 0) {
    g.cbase[cnt] = total;
    g.m = cnt;
    g.nt = total * Q;
    g.gid = gid;
  }
  const int nt = total * Q;
  const double* Tg = a.grec + a.grp_toff[gid];
  if (nt <= kGroupSmemTrace)
    for (int t = lane; t < nt * nt; t += 32) g.tinv[t] = Tg[t];
  __syncwarp();
}

template <int P>
__device__ __forceinline__ void adj_group_direct(const AdjArgs& a, int d, int s0, AdjGroupSmem<P>& g) {
  constexpr int Q = P + 1, N = Q * Q;
  using L = Rec<P, double>;
  const int lane = threadIdx.x & 31;
  const int first = a.slot_first[s0];
  const int m = g.m, nt = g.nt;
  // g~: w_d g minus the couplings from receivers outside the group
  for (int idx = lane; idx < m * N; idx += 32) {
    const int mi = idx / N, i = idx % N;
    const uint4 info = g.info[mi];
    const int e = (int)info.x;
    const unsigned bits = info.y;
    double r = a.weights[d] * a.g[(size_t)e * N + i];
    const int ia = i % Q, ib = i / Q;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!((bits >> (8 + f)) & 1u) || ((bits >> (4 + f)) & 1u)) continue;   // no external receiver
      const int t = f == 0 ? (ib == 0 ? ia : -1) : f == 1 ? (ia == P ? ib : -1)
                  : f == 2 ? (ib == P ? ia : -1) : (ia == 0 ? ib : -1);
      if (t < 0) continue;
      const uint32_t lk = a.link[(long long)(first + mi) * 4 + f];
      if (lk == ~0u) continue;
      const long long mn = (long long)(lk >> 2);
      const double* W = L::slot(L::s_at(a.rec, mn), L::x_at(a.recx, mn), (int)(lk & 3u)) + t * N;
      const double* rn = a.radj + ((size_t)d * a.E + nb_elem(a.nx, a.ny, e, f)) * N;
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) s += W[j] * rn[j];
      r -= s;
    }
    g.z[idx] = r;
  }
  __syncwarp();
  // v = W^T g~ over the internal couplings: v_(c,t) = sum_i W_(a,f)[t][i] g~_a[i]
  for (int j = lane; j < nt; j += 32) {
    const uint32_t cp = g.cpl[j / Q];
    const int am = (int)(cp & 0xffu), t = j % Q;
    const double* W = L::slot(L::s_at(a.rec, first + am), L::x_at(a.recx, first + am), (int)(cp >> 24)) + t * N;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) s += W[i] * g.z[am * N + i];
    g.v[j] = s;
  }
  __syncwarp();
  // w = T^T v (column r of T is contiguous)
  const double* Tm = nt <= kGroupSmemTrace ? g.tinv : a.grec + a.grp_toff[g.gid];
  for (int rr = lane; rr < nt; rr += 32) {
    double acc0 = 0.0, acc1 = 0.0;
    int j = 0;
    for (; j + 1 < nt; j += 2) {
      acc0 += Tm[rr * nt + j] * g.v[j];
      acc1 += Tm[rr * nt + j + 1] * g.v[j + 1];
    }
    if (j < nt) acc0 += Tm[rr * nt + j] * g.v[j];
    g.w[rr] = acc0 + acc1;
  }
  __syncwarp();
  // r = g~ - P^T w: the trace unknown (c, t) is node t of face opp(f) of neighbour b
  for (int idx = lane; idx < m * N; idx += 32) {
    const int mi = idx / N, i = idx % N;
    double r = g.z[idx];
    const int ntc = nt / Q;
    for (int c = 0; c < ntc; ++c) {
      const uint32_t cp = g.cpl[c];
      if ((int)((cp >> 16) & 0xffu) != mi) continue;
      const int fo = ((int)((cp >> 8) & 0xffu) + 2) & 3;
#pragma unroll
      for (int t = 0; t < Q; ++t)
        if (face_dof<P>(fo, t) == i) r -= g.w[c * Q + t];
    }
    a.radj[((size_t)d * a.E + g.info[mi].x) * N + i] = r;
  }
  __syncwarp();
}

// ------------------------------------------------------------ single-CTA backward sweep
// One CTA of 16 warps per direction walks the forward schedule's levels backwards.  The
// couplings are the forward ones with the roles swapped: a receiver e' (done first)
// projects its r onto the face of each donor that feeds one of its staged W slots,
// s_t = sum_i W[t][i] r_i (the C^T lambda term of the donor's face nodes), and writes the
// p+1 values into the slot through which the forward sweep passed the donor's face values;
// the donor subtracts them from w_d g on its outflow face rows.  Warp 15 streams the
// singles' records (info + W slots 0, 1), their w_d g rows and slot ids through a ring of
// chunk buffers (bulk copies); warps 0..11 compute rounds of 12 SPC tasks, the
// projections summed over a task's rows through a per-warp scratch; warps 12..14 run the
// coupled groups (inner iteration on the transposed blocks); a named barrier separates
// levels.  Couplings whose slot is missing (receivers in groups, third and fourth W
// slots, capacity) are read from global memory (slot-id flag bit 1).
template <int P>
struct AdjShape {
  static constexpr int Q = P + 1, N = Q * Q;
  using L = Rec<P, double>;
  static constexpr int kCompute = 12, kGroupWarps = 3, kProducer = 15, kThreads = 512;
  static constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  static constexpr int CH = kCompute * SPC;
  static constexpr int kTaskBytes = L::kStaged + L::kYBytes + 16;
  static constexpr int RC = (48 * 1024) / (CH * kTaskBytes) > 8 ? 8
                          : ((48 * 1024) / (CH * kTaskBytes) < 1 ? 1 : (48 * 1024) / (CH * kTaskBytes));
  static constexpr int CK = RC * CH;
  static constexpr int kYOff = CK * L::kStaged;
  static constexpr int kTsOff = kYOff + CK * L::kYBytes;
  static constexpr int kRound = kTsOff + CK * 16;
  static constexpr int kMaxRing = 16;
  static constexpr int kBars = 2 * kMaxRing * 8;
  static constexpr int kScratch = kCompute * SPC * 2 * Q * N * 8;   // per warp [task][slot][t][row]
  static constexpr int kGs = ((int)sizeof(AdjGroupSmem<P>) + 15) / 16 * 16;
  static constexpr int kGroup = kGroupWarps * kGs;
  static constexpr int kSmemMax = 227 * 1024;
  static constexpr int avail() { return kSmemMax - kBars - kScratch - kGroup; }
};

__global__ void adj_yadj_kernel(long long nmem, int n, int ystride, long long E, const uint32_t* __restrict__ code,
                                const double* __restrict__ weights, const double* __restrict__ g,
                                double* __restrict__ y) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= nmem * n) return;
  const long long m = t / n;
  const int i = (int)(t - m * n);
  const uint32_t c = code[m];
  const int d = (int)(c >> 22), e = (int)(c & 0x3fffffu);
  y[m * ystride + i] = weights[d] * g[(size_t)e * n + i];
}

template <int P>
__global__ void __maxnreg__(128) adjoint_cta_kernel(AdjArgs a) {
  using Sh = AdjShape<P>;
  using L = Rec<P, double>;
  constexpr int Q = P + 1, N = Q * Q, SPC = Sh::SPC, CH = Sh::CH, CK = Sh::CK;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char adj_smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(adj_smem);
  uint64_t* empty = full + Sh::kMaxRing;
  double* scratch_all = reinterpret_cast<double*>(adj_smem + Sh::kBars);
  unsigned char* gsm_all = adj_smem + Sh::kBars + Sh::kScratch;
  double* tr = reinterpret_cast<double*>(adj_smem + Sh::kBars + Sh::kScratch + Sh::kGroup);
  unsigned char* ring = adj_smem + Sh::kBars + Sh::kScratch + Sh::kGroup + a.tr_bytes;
  const unsigned NB = (unsigned)a.ring;
  const int d = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (unsigned b = 0; b < NB; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], Sh::kCompute);
    }
    mbar_fence_init();
  }
  __syncthreads();
  const int k0 = a.dir_lev0[d], k1 = a.dir_lev0[d + 1];
  // level tables of levels kt - j (lane j) and kt - 32 - j, read with shuffles, walking down
  int kt = k1 - 1;
  int lb0, le0, lg0, lm0, lb1, le1, lg1, lm1;
  auto load_win = [&](int top, int& lb, int& le, int& lg, int& lm) {
    const int kk = top - lane;
    const bool ok = kk >= k0;
    lb = ok ? a.lev_begin[kk] : 0;
    le = ok ? a.lev_begin[kk + 1] : 0;
    lg = ok ? a.lev_gbegin[kk] : 0;
    lm = ok ? a.lev_mbegin[kk] : 0;
  };
  load_win(kt, lb0, le0, lg0, lm0);
  load_win(kt - 32, lb1, le1, lg1, lm1);
  auto lev = [&](int kk, int x0, int x1) { const int j = kt - kk; return __shfl_sync(FULL, j < 32 ? x0 : x1, j & 31); };
  auto advance = [&](int k) {
    if (kt - k >= 32) {
      kt -= 32;
      lb0 = lb1; le0 = le1; lg0 = lg1; lm0 = lm1;
      load_win(kt - 32, lb1, le1, lg1, lm1);
    }
  };
  // producer waits (a buffer released, copies drained) do not stop on the status bit
  auto bounded_wait = [&](uint64_t* bar, unsigned parity) {
    uint32_t n = 0;
    while (!mbar_try_wait(bar, parity) && ++n < kAdjWaitIters) {
    }
    if (n >= kAdjWaitIters) atomicOr(a.status, kDevTimeout);
  };
  // consumer waits for a staged chunk give up early on the status bit; a warp whose wait
  // gave up never reads a staged chunk again but still releases every buffer and reaches
  // every level barrier
  bool failed = false;
  auto data_wait = [&](uint64_t* bar, unsigned parity) {
    const bool ok = mbar_wait_data(bar, parity, kAdjWaitIters, a.status);
    if (!ok) atomicOr(a.status, kDevTimeout);
    failed = failed || __any_sync(0xffffffffu, !ok);
  };
  auto next = [&](unsigned& b, unsigned& par) {
    if (++b == NB) { b = 0; par ^= 1u; }
  };

  if (warp == Sh::kProducer) {
    unsigned rc = 0, b = 0, par = 0;
    for (int k = k1 - 1; k >= k0; --k) {
      advance(k);
      const int nsingle = lev(k, lg0, lg1) - lev(k, lb0, lb1), mb = lev(k, lm0, lm1);
      for (int r0 = 0; r0 < nsingle; r0 += CK, ++rc, next(b, par)) {
        if (lane != 0) continue;
        if (rc >= NB) bounded_wait(&empty[b], par ^ 1u);
        const int cnt = min(CK, nsingle - r0);
        const long long m0 = (long long)mb + r0;
        unsigned char* rb = ring + (size_t)b * Sh::kRound;
        fence_proxy_async_smem();
        if (!(VEF_IN_RANGE(m0, a.nmem, a.status) && VEF_IN_RANGE(m0 + cnt - 1, a.nmem, a.status))) {
          mbar_arrive_expect_tx(&full[b], 0u);   // the round completes without data
          continue;
        }
        mbar_arrive_expect_tx(&full[b], (unsigned)(cnt * (L::kStaged + L::kYBytes + 16)));
        bulk_g2s(rb, L::s_at(a.rec, m0), (unsigned)(cnt * L::kStaged), &full[b]);
        bulk_g2s(rb + Sh::kYOff, a.yadj + m0 * L::kYStride, (unsigned)(cnt * L::kYBytes), &full[b]);
        bulk_g2s(rb + Sh::kTsOff, a.tslot + m0, (unsigned)(cnt * 16), &full[b]);
      }
    }
    if (lane == 0)
      for (unsigned j = rc > NB ? rc - NB : 0u; j < rc; ++j) bounded_wait(&full[j % NB], (j / NB) & 1u);
    return;
  }

  const bool compute = warp < Sh::kCompute;
  const int i = lane % N, s_lane = lane / N;
  const int task = warp * SPC + s_lane;
  const bool lane_ok = compute && lane < SPC * N;
  // the faces dof row i lies on (two at a corner) and its node position on each
  const int ia = i % Q, ib = i / Q;
  int fA = -1, pA = 0, fB = -1, pB = 0;
  auto on_face = [&](int f, int pos) {
    if (fA < 0) { fA = f; pA = pos; } else { fB = f; pB = pos; }
  };
  if (ib == 0) on_face(0, ia);
  if (ia == P) on_face(1, ib);
  if (ib == P) on_face(2, ia);
  if (ia == 0) on_face(3, ib);
  double* scratch = scratch_all + (compute ? warp : 0) * (SPC * 2 * Q * N);
  double* radj = a.radj + (size_t)d * a.E * N;
  const int ntr = a.tr_bytes / (Q * (int)sizeof(double));   // trace slots in shared memory
  (void)ntr;
  if (threadIdx.x < Q) tr[kTraceZero * Q + threadIdx.x] = 0.0;
  const int gidx = warp - Sh::kCompute;
  AdjGroupSmem<P>& gs = *reinterpret_cast<AdjGroupSmem<P>*>(gsm_all + (compute ? 0 : gidx) * Sh::kGs);
  auto direct = [&](int slot) { return a.slot_gid != nullptr && a.slot_gid[slot] >= 0; };
  unsigned rb_i = 0, rpar = 0;
  named_barrier(1, (Sh::kCompute + Sh::kGroupWarps) * 32);   // the zero trace is in place
  for (int k = k1 - 1; k >= k0; --k) {
    advance(k);
    const int sb = lev(k, lb0, lb1), sg = lev(k, lg0, lg1), se = lev(k, le0, le1), mb = lev(k, lm0, lm1);
    if (compute) {
      const int nsingle = sg - sb;
      for (int c0 = 0; c0 < nsingle; c0 += CK) {
        const unsigned char* rb = ring + (size_t)rb_i * Sh::kRound;
        data_wait(&full[rb_i], rpar);
        const int cend = min(CK, nsingle - c0);
        for (int tk0 = 0; tk0 < cend; tk0 += CH) {   // the chunk's rounds
          const int tk = tk0 + task;
          const bool act = !failed && lane_ok && tk < cend;
          double r = 0.0;
          uint4 ts = make_uint4(0u, 0u, 0u, 0u);
          const char* rs = (const char*)rb;
          if (act) {
            rs = (const char*)rb + tk * L::kStaged;
            const uint4 info = *reinterpret_cast<const uint4*>(rs);
            ts = *reinterpret_cast<const uint4*>(rb + Sh::kTsOff + tk * 16);
            r = reinterpret_cast<const double*>(rb + Sh::kYOff + tk * L::kYBytes)[i];
            // the receivers' projections on this row's faces (no slot: kTraceSink -> zero)
            auto rd = [&](int f) {
              if (f < 0) return kTraceZero;
              const unsigned id = ((f >= 2 ? ts.z : ts.y) >> (16 * (f & 1))) & 0xffffu;
              return id == kTraceSink || !VEF_IN_RANGE(id, ntr, a.status) ? kTraceZero : id;
            };
            r -= tr[rd(fA) * Q + pA];
            r -= tr[rd(fB) * Q + pB];
            const int e = (int)info.x;
            if (ts.w & 2u) {   // rare: a receiver's projection read from global memory
              const long long m = (long long)mb + c0 + tk;
#pragma unroll 1
              for (int f = 0; f < 4; ++f) {
                if (!((info.y >> (8 + f)) & 1u)) continue;
                if ((((f >= 2 ? ts.z : ts.y) >> (16 * (f & 1))) & 0xffffu) != kTraceSink) continue;
                const int t = f == fA ? pA : (f == fB ? pB : -1);
                if (t < 0) continue;
                const uint32_t lk = a.link[m * 4 + f];
                if (lk == ~0u) continue;
                const long long mn = (long long)(lk >> 2);
                if (!(VEF_IN_RANGE(mn, a.nmem, a.status) && VEF_IN_RANGE(nb_elem(a.nx, a.ny, e, f), a.E, a.status)))
                  continue;
                const double* W = L::slot(L::s_at(a.rec, mn), L::x_at(a.recx, mn), (int)(lk & 3u)) + t * N;
                const double* rn = radj + (size_t)nb_elem(a.nx, a.ny, e, f) * N;
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < N; ++j) acc += W[j] * rn[j];
                r -= acc;
              }
            }
            if (VEF_IN_RANGE(e, a.E, a.status)) radj[(size_t)e * N + i] = r;
            // this task's projections onto its donors' faces, W slots 0 and 1 (zero slots
            // of absent faces give zero products)
            const double* W = L::slot(rs, nullptr, 0);
#pragma unroll
            for (int sl = 0; sl < 2; ++sl)
#pragma unroll
              for (int t = 0; t < Q; ++t)
                scratch[((s_lane * 2 + sl) * Q + t) * N + i] = W[sl * L::kSlot + t * N + i] * r;
          }
          __syncwarp();
          for (int q = lane; !failed && q < SPC * 2 * Q; q += 32) {
            const int s = q / (2 * Q), sl = (q / Q) % 2, t = q % Q;
            const int tks = tk0 + warp * SPC + s;
            if (tks >= cend) continue;
            const uint4 tss = *reinterpret_cast<const uint4*>(rb + Sh::kTsOff + tks * 16);
            const unsigned wid = (tss.x >> (16 * sl)) & 0xffffu;
            if (wid == kTraceZero || !VEF_IN_RANGE(wid, ntr, a.status)) continue;
            const double* pr = scratch + ((s * 2 + sl) * Q + t) * N;
            double sum = 0.0;
#pragma unroll
            for (int j = 0; j < N; ++j) sum += pr[j];
            tr[wid * Q + t] = sum;
          }
          __syncwarp();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[rb_i]);
        next(rb_i, rpar);
      }
    } else {
      for (int g = sg + gidx; g < se; g += Sh::kGroupWarps) {
        if (direct(g)) {
          adj_group_stage<P>(a, g, gs);
          adj_group_direct<P>(a, d, g, gs);
        } else {
          adj_group<P, false>(a, d, g);
        }
      }
    }
    named_barrier(1, (Sh::kCompute + Sh::kGroupWarps) * 32);
  }
}

// lambda = A^{-T} r and the gradient sums for every (element, direction) once the
// backward sweep has produced all r: nothing downstream needs them, so they stay off the
// sweep's level-by-level critical path.  One lane per dof row, SPC tasks per warp.
template <int P>
__global__ void __launch_bounds__(128) adj_finish_kernel(AdjArgs a) {
  constexpr int N = (P + 1) * (P + 1);
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  const int lane = threadIdx.x & 31;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long mm = gw * SPC + lane / N;
  const int i = lane % N;
  const bool valid = lane < SPC * N && mm < a.nmem;
  const long long m = valid ? mm : 0;
  const uint32_t c = a.code[m];
  const int d = (int)(c >> 22), e = (int)(c & 0x3fffffu);
  const double r = valid ? a.radj[((size_t)d * a.E + e) * N + i] : 0.0;
  adj_finish<P>(a, m, d, e, i, valid, r);
}

// Receiver links of the backward sweep: for member m = (d, e) and a face f across which
// e feeds its neighbour, the neighbour's member index and the W slot it holds for the
// face toward e (its slots are its interior inflow faces in face order).
__global__ void adj_link_kernel(long long nmem, long long E, int nx, int ny, const uint32_t* __restrict__ code,
                                const uint16_t* __restrict__ finfo, const int* __restrict__ member_of,
                                uint32_t* __restrict__ link) {
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= nmem) return;
  const uint32_t c = code[m];
  const int d = (int)(c >> 22), e = (int)(c & 0x3fffffu);
  const uint16_t bits = finfo[(size_t)d * E + e];
  for (int f = 0; f < 4; ++f) {
    uint32_t lk = ~0u;
    const int nb = nb_elem(nx, ny, e, f);
    if ((bits & (1u << (8 + f))) && nb >= 0) {
      const uint16_t nbits = finfo[(size_t)d * E + nb];
      const int fn = (f + 2) & 3;
      int slot = 0;
      for (int g = 0; g < fn; ++g)
        if ((nbits & (1u << g)) && nb_elem(nx, ny, nb, g) >= 0) ++slot;
      if (nbits & (1u << fn)) lk = ((uint32_t)member_of[(size_t)d * E + nb] << 2) | (uint32_t)slot;
    }
    link[m * 4 + f] = lk;
  }
}

__global__ void mvec_kernel(long long E, int n, const double* __restrict__ M,
                            const double* __restrict__ x, double* __restrict__ y) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= E * n) return;
  long long e = t / n;
  int i = (int)(t % n);
  double s = 0.0;
  for (int j = 0; j < n; ++j) s += M[(e * n + i) * n + j] * x[e * n + j];
  y[t] = s;
}

static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// forward factorisation (FP64) from sweep.cu
vef_status factor_fp64(Mesh* mesh, Schedule* S, const double* sigma_t, cudaStream_t stream);
vef_status collect_status(Mesh& M, cudaStream_t stream, vef_info* info);

template <int P>
static vef_status launch_adjoint(Mesh& M, AdjArgs a, int D, int cs, int warps, cudaStream_t s);

template <int P>
static vef_status launch_adjoint_cta(Mesh& M, Schedule& S, AdjArgs a, cudaStream_t s) {
  using Sh = AdjShape<P>;
  using L = Rec<P, double>;
  constexpr int N = (P + 1) * (P + 1);
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  vef_status st = ensure_buffer(&M.ybuf, &M.ybuf_cap, (size_t)S.members * L::kYBytes);
  if (st != VEF_OK) return st;
  a.recx = (const double*)((const char*)a.rec + a.nmem * (long long)L::kStaged);
  a.yadj = (const double*)M.ybuf;
  a.tslot = S.tslot;
  a.tr_bytes = (S.trace_slots * (P + 1) * 8 + 15) / 16 * 16;
  a.ring = std::min(Sh::kMaxRing, (Sh::avail() - a.tr_bytes) / Sh::kRound);
  if (a.ring < 2) return launch_adjoint<P>(M, a, S.D, 8, 4, s);   // slots too many: cluster sweep
  const size_t smem = (size_t)Sh::kBars + Sh::kScratch + Sh::kGroup + a.tr_bytes + (size_t)a.ring * Sh::kRound;
  if (!S.ngroups || !S.grec64) a.slot_gid = nullptr;   // every group by the inner iteration
  a.member_nbpos = S.member_nbpos;
  a.grp_toff = S.grp_toff;
  a.grec = (const double*)S.grec64;
  {
    KTimer kt(&M, VEF_K_SOURCE, s);
    adj_yadj_kernel<<<nblk(a.nmem * N, 256), 256, 0, s>>>(a.nmem, N, L::kYStride, a.E, a.code, a.weights, a.g,
                                                          (double*)M.ybuf);
    VEF_CUDA_TRY(cudaGetLastError());
  }
  VEF_CUDA_TRY(cudaFuncSetAttribute(adjoint_cta_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  KTimer kt(&M, VEF_K_ADJOINT, s);   // the backward sweep and the gradient post-pass
  adjoint_cta_kernel<P><<<(unsigned)S.D, Sh::kThreads, smem, s>>>(a);
  VEF_CUDA_TRY(cudaGetLastError());
  const long long nwarp = (a.nmem + SPC - 1) / SPC;
  adj_finish_kernel<P><<<nblk(nwarp * 32, 128), 128, 0, s>>>(a);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}

template <int P>
static vef_status launch_adjoint(Mesh& M, AdjArgs a, int D, int cs, int warps, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(D * cs));
  cfg.blockDim = dim3((unsigned)(32 * warps));
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cs > 8)
    VEF_CUDA_TRY(cudaFuncSetAttribute(adjoint_kernel<P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  a.cluster_size = cs;
  a.recx = (const double*)((const char*)a.rec + a.nmem * (long long)Rec<P, double>::kStaged);
  KTimer kt(&M, VEF_K_ADJOINT, s);
  VEF_CUDA_TRY(cudaLaunchKernelEx(&cfg, adjoint_kernel<P>, a));
  constexpr int N = (P + 1) * (P + 1);
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  const long long nwarp = (a.nmem + SPC - 1) / SPC;
  adj_finish_kernel<P><<<nblk(nwarp * 32, 128), 128, 0, s>>>(a);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}

}  // namespace vef

using namespace vef;

extern "C" vef_status vef_adjoint_sweep(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                                        const double* phi_in, const double* omega,
                                        const double* weights, int D, const double* psi_ckpt,
                                        const double* g, double* lambda, double* dR_dsigma_t,
                                        double* dR_dsigma_s, const vef_opts* opts, vef_info* info,
                                        void* stream) {
  if (!mesh || !sigma_t || !omega || !weights || !psi_ckpt || !g || !dR_dsigma_t) {
    set_last_error("mesh, sigma_t, omega, weights, psi_ckpt, g, dR_dsigma_t are required");
    return VEF_ERR_INVALID_ARG;
  }
  if (phi_in && (!sigma_s || !dR_dsigma_s)) {
    set_last_error("phi_in given: sigma_s and dR_dsigma_s are required");
    return VEF_ERR_INVALID_ARG;
  }
  if (D < 1 || D > kMaxD) { set_last_error("D must be in 1..1023"); return VEF_ERR_INVALID_ARG; }
  Mesh& M = mesh->impl;
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != M.device) { set_last_error("mesh belongs to another device"); return VEF_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  vef_status st;
  Schedule* S = get_schedule(&M, omega, weights, D, s, &st);
  if (!S) return st;
  if ((st = factor_fp64(&M, S, sigma_t, s)) != VEF_OK) return st;
  if (!S->adj_link) {
    if (S->members >= (1LL << 30)) {
      set_last_error("adjoint sweep supports at most 2^30 (element, direction) pairs");
      return VEF_ERR_INVALID_ARG;
    }
    size_t cap = 0;
    if ((st = ensure_buffer((void**)&S->adj_link, &cap, (size_t)S->members * 4 * sizeof(uint32_t))) != VEF_OK)
      return st;
    adj_link_kernel<<<nblk(S->members, 256), 256, 0, s>>>(S->members, M.E, M.nx, M.ny, S->member_code,
                                                          S->faceinfo, S->member_of, S->adj_link);
    VEF_CUDA_TRY(cudaGetLastError());
  }
  const long long tot = (long long)D * M.E * M.n;
  const size_t need = (size_t)tot * sizeof(double) * (lambda ? 1 : 2) + (size_t)M.E * M.n * sizeof(double);
  if ((st = ensure_buffer((void**)&M.work2, &M.work2_cap, need)) != VEF_OK) return st;
  AdjArgs a{};
  a.dir_lev0 = S->dir_lev0;
  a.lev_begin = S->lev_begin;
  a.lev_gbegin = S->lev_gbegin;
  a.lev_mbegin = S->lev_mbegin;
  a.slot_gid = S->slot_gid;
  a.slot_first = S->slot_first;
  a.slot_count = S->slot_count;
  a.code = S->member_code;
  a.member_of = S->member_of;
  a.finfo = S->faceinfo;
  a.omega = S->omega_dev;
  a.weights = S->weights_dev;
  a.rec = (const double*)S->rec64;
  a.nmem = S->members;
  a.g = g;
  if (opts && (opts->flags & VEF_CKPT_FP32)) a.psi32 = reinterpret_cast<const float*>(psi_ckpt);
  else a.psi = psi_ckpt;
  a.Mm = M.Mmat;
  a.radj = M.work2;
  a.lambda = lambda ? lambda : M.work2 + tot;
  double* mphi = M.work2 + tot * (lambda ? 1 : 2);
  a.mphi = phi_in ? mphi : nullptr;
  a.link = S->adj_link;
  a.dst = dR_dsigma_t;
  a.dss = dR_dsigma_s;
  a.status = M.dev_status;
  a.nx = M.nx;
  a.ny = M.ny;
  a.E = M.E;
  const int maxp = (opts && opts->max_passes > 0) ? opts->max_passes : 8;
  a.tol = (opts && opts->tol > 0.0) ? std::max(opts->tol, 2e-15) : 2e-15;
  a.max_inner = std::max(2, 4 * maxp);
  if (phi_in) {
    KTimer kt(&M, VEF_K_SOURCE, s);
    mvec_kernel<<<nblk(M.E * M.n, 256), 256, 0, s>>>(M.E, M.n, M.Mmat, phi_in, mphi);
  }
  VEF_CUDA_TRY(cudaMemsetAsync(dR_dsigma_t, 0, M.E * sizeof(double), s));
  if (dR_dsigma_s) VEF_CUDA_TRY(cudaMemsetAsync(dR_dsigma_s, 0, M.E * sizeof(double), s));
  const int tile = (opts && opts->tile_override > 0) ? opts->tile_override : 804;
  const int cs = std::min(16, std::max(1, tile / 100)), warps = std::min(8, std::max(1, tile % 100));
  // one CTA per direction unless the caller asks for the cluster sweep
  const bool cta = !(opts && (opts->tile_override > 0 || (opts->flags & VEF_SWEEP_CLUSTER)));
  switch (M.p) {
    case 1: st = cta ? launch_adjoint_cta<1>(M, *S, a, s) : launch_adjoint<1>(M, a, D, cs, warps, s); break;
    case 2: st = cta ? launch_adjoint_cta<2>(M, *S, a, s) : launch_adjoint<2>(M, a, D, cs, warps, s); break;
    case 3: st = cta ? launch_adjoint_cta<3>(M, *S, a, s) : launch_adjoint<3>(M, a, D, cs, warps, s); break;
    default: st = cta ? launch_adjoint_cta<4>(M, *S, a, s) : launch_adjoint<4>(M, a, D, cs, warps, s); break;
  }
  if (st != VEF_OK) return st;
  if (info) {
    info->passes = 1;
    info->rel_residual = -1.0;
    info->coupled_groups = S->coupled_groups;
    info->lagged_face_points = S->lagged_points;
    info->levels = S->levels;
    return collect_status(M, s, info);
  }
  return VEF_OK;
}
