// Transport sweep: dependency-free right-hand-side apply, wavefront solve (one CTA per
// direction, also for batches; one cluster per direction on request or when the batch tuner
// picks it), FP64 residual and mixed-precision defect correction, and source iteration.
//
// The element equations (upwind DG, pointwise upwinding at face Gauss points) give, for
// direction d and element e,
//     A_{e,d} psi_e = b_e - sum_{inflow faces f} Cin_{f} u_f,
//     A_{e,d} = sigma_t M_e - mu Gx_e - eta Gy_e + sum_f sum_k max(c_k, 0) l_a(s_k) l_b(s_k),
//     (Cin_f)_{a t} = sum_k min(c_k, 0) l_a(s_k) l_t(s_k),   c_k = w_k Omega . (n ds)_k,
// with u_f the upwind neighbour's face-node values (GLL basis: its trace on the shared face
// is spanned by its p+1 face nodes).  Only the u_f terms depend on other elements.
//
// factor_kernel (factor_impl.cuh) stores per (element, direction) A^{-1} and
// W_f = A^{-1} Cin_f.  y = A^{-1} b is formed for every (element, direction) with no
// dependencies: by apply workers inside the sweep launch when the directions leave SMs
// free (apply_worker), else by apply_kernel before it.  The wavefront kernels
// (sweep_cta_kernel, sweep_kernel) then only compute psi = y - sum_f W_f u_f along the
// dependency levels, one lane per dof row, so the chain of dependent work per level is a
// few FMAs (on this GPU a warp-wide FP64 FMA occupies its SM sub-partition for ~64
// cycles, so per-element latency, not total flops, bounds a wavefront).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <cstdio>

#include "device.cuh"

namespace vef {



// ----------------------------------------------------------------- right-hand sides
// bvol[e][i] = sum_j M_ij (sigma_s phi_in_j / (4 pi) + q_j)  (isotropic, direction-free)
__global__ void bvol_kernel(long long E, int n, const double* __restrict__ M,
                            const double* __restrict__ sigma_s, const double* __restrict__ phi_in,
                            const double* __restrict__ q, double* __restrict__ bvol) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= E * n) return;
  long long e = t / n;
  int i = (int)(t % n);
  const double ss = phi_in ? sigma_s[e] / kFourPi : 0.0;
  double s = 0.0;
  for (int j = 0; j < n; ++j) {
    double v = 0.0;
    if (phi_in) v += ss * phi_in[e * n + j];
    if (q) v += q[e * n + j];
    s += M[(e * n + i) * n + j] * v;
  }
  bvol[t] = s;
}

// --------------------------------------------------------------------------- sweep
template <typename T>
struct SweepArgs {
  const int* dir_lev0;
  const int* lev_begin;
  const int* lev_gbegin;
  const int* lev_mbegin;
  const uint2* member_info;
  const uint32_t* member_nbpos;
  int cluster_size;
  const int* slot_first;
  const int* slot_count;
  const int* slot_gid;       // group index of a directly solved group slot, or -1; null = none
  const long long* grp_toff; // offset of each group's trace-system inverse in grec
  const T* grec;
  const uint32_t* code;
  const int* member_of;
  const uint16_t* finfo;
  const double* omega;
  const T* rec;             // staged record array S (see Rec)
  const T* recx;            // extra record array X
  const double* bvol;      // [E][n] (mode 0)
  const double* src_aniso; // [D][E][n] or null (mode 0)
  const double* Mm;        // FP64 mass matrices (anisotropic source)
  const double* inflow;    // [D][nbf][nq] or null (mode 0)
  const T* nds;            // [E][4][nq][2]
  const double* rhs;       // [D][E][n] (mode 1)
  T* out;                  // [D][E][n]
  T* y;                    // [D][E][n] A^{-1} b (apply_kernel or the apply workers)
  unsigned int* status;    // [0] status bits, [2] max inner iterations
  const uint4* tslot;      // single-CTA sweep: trace slot ids per member (Schedule::tslot)
  int* ready;              // single-CTA sweep with fused apply: [nd][bands] band done flags
  int nd;                  //   direction CTAs (the others apply A^{-1})
  int bands;               //   bands per direction (kApplyBand levels each)
  long long nmem;          //   members of the schedule
  int ring;                // single-CTA sweep: round buffers in the ring
  int tr_bytes;            // single-CTA sweep: bytes of the trace slots
  int nx, ny;
  long long E, nbf;
  T tol;
  int max_inner;
  FaceTab<T> ft;
};

// own right-hand-side entry b_i of (d, e): volume source plus boundary inflow (mode 0),
// or the given residual (mode 1)
template <int P, typename T, int MODE>
__device__ __forceinline__ T rhs_entry(const SweepArgs<T>& a, int d, int e, int i, uint16_t bits,
                                       T mu, T eta) {
  constexpr int Q = P + 1, N = Q * Q, NQ = P + 2;
  if (MODE == 1) return (T)a.rhs[((size_t)d * a.E + e) * N + i];
  double b = a.bvol[(size_t)e * N + i];
  if (a.src_aniso) {
    const double* Mr = a.Mm + ((size_t)e * N + i) * N;
    const double* qd = a.src_aniso + ((size_t)d * a.E + e) * N;
#pragma unroll
    for (int j = 0; j < N; ++j) b += Mr[j] * qd[j];
  }
  T bt = (T)b;
  if (a.inflow) {
    const int ia = i % Q, ib = i / Q;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!(bits & (1u << f))) continue;
      if (nb_elem(a.nx, a.ny, e, f) >= 0) continue;
      int pos = -1;
      if (f == 0 && ib == 0) pos = ia;
      if (f == 1 && ia == P) pos = ib;
      if (f == 2 && ib == P) pos = ia;
      if (f == 3 && ia == 0) pos = ib;
      if (pos < 0) continue;
      const int bf = bface(a.nx, a.ny, e, f);
      const double* pb = a.inflow + ((size_t)d * a.nbf + bf) * NQ;
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        const T* v = a.nds + (((size_t)e * 4 + f) * NQ + k) * 2;
        const T s = a.ft.w[k] * (mu * v[0] + eta * v[1]);
        if (s < (T)0) bt -= s * (T)pb[k] * a.ft.l[pos][k];
      }
    }
  }
  return bt;
}

// y = A^{-1} b for every (element, direction): no dependencies, one lane per dof row,
// records read in schedule order (consecutive members are adjacent in memory); y rows are
// written in schedule order with a 16-byte-aligned stride.
// one warp: tasks [m0, m0 + SPC) of those below mend (all lanes of the warp take part)
template <int P, typename T, int MODE>
__device__ __forceinline__ void apply_warp(const SweepArgs<T>& a, long long m0, long long mend) {
  constexpr int Q = P + 1, N = Q * Q;
  using L = Rec<P, T>;
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  constexpr unsigned FULL = 0xffffffffu;
  (void)Q;
  const int lane = threadIdx.x & 31;
  const long long m = m0 + lane / N;
  const int i = lane % N;
  const bool valid = (lane < SPC * N) && (m < mend);
  T bi = 0;
  if (valid) {
    const uint32_t cd = a.code[m];
    const int d = (int)(cd >> 22);
    const int e = (int)(cd & 0x3fffffu);
    const uint16_t bits = a.finfo[(size_t)d * a.E + e];
    bi = rhs_entry<P, T, MODE>(a, d, e, i, bits, (T)a.omega[2 * d], (T)a.omega[2 * d + 1]);
  }
  const T* ai = L::ainv(L::x_at(a.recx, valid ? m : 0));
  const int base = (lane / N) * N;
  T y = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const T bj = __shfl_sync(FULL, bi, (base + j) & 31);
    if (valid) y += ai[j * N + i] * bj;
  }
  if (valid) a.y[(size_t)m * L::kYStride + i] = y;
}

template <int P, typename T, int MODE>
__global__ void __launch_bounds__(128) apply_kernel(SweepArgs<T> a, long long nmem) {
  constexpr int N = (P + 1) * (P + 1);
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  apply_warp<P, T, MODE>(a, gw * SPC, nmem);
}

// upwind correction of row i for face f of member record r: sum_t W_f[t][i] u_t
// (CG: the neighbour's values are read at L2, as a cluster's other CTAs wrote them; the
// single-CTA sweep reads them with ordinary loads)
template <int P, typename T, bool CG = true>
__device__ __forceinline__ T face_term(const T* W, const T* un, int f, int i) {
  constexpr int Q = P + 1, N = Q * Q;
  T acc = 0;
#pragma unroll
  for (int t = 0; t < Q; ++t) {
    const T* up = un + face_dof<P>((f + 2) & 3, t);
    acc += W[t * N + i] * (CG ? ldcg(up) : *up);
  }
  return acc;
}

// Coupled group by inner block Gauss-Seidel over its members, in global memory (groups
// beyond the direct limits, or every group when the caller asks for the iteration).
template <int P, typename T, int MODE, bool CG = true>
__device__ __forceinline__ void group_solve(const SweepArgs<T>& a, int d, int s0) {
  constexpr int Q = P + 1, N = Q * Q;
  using L = Rec<P, T>;
  constexpr unsigned FULL = 0xffffffffu;
  (void)Q;
  const int lane = threadIdx.x & 31;
  const int first = a.slot_first[s0];
  const int cnt = a.slot_count[s0];
  if (!(VEF_IN_RANGE(first, a.nmem, a.status) && VEF_IN_RANGE(first + cnt - 1, a.nmem, a.status))) return;
  const int i = lane;
  const bool act = lane < N;
  int it = 0;
  bool conv = false;
  for (; it < a.max_inner; ++it) {
    T dmax = 0, amax = 0;
    for (int mi = 0; mi < cnt; ++mi) {
      const char* r = L::s_at(a.rec, first + mi);
      const char* rx = L::x_at(a.recx, first + mi);
      const uint4 info = *reinterpret_cast<const uint4*>(r);
      const int e = (int)info.x;
      const unsigned bits = info.y;
      if (act) {
        T y = ldcg(a.y + (size_t)(first + mi) * L::kYStride + i);
        for (int f = 0; f < 4; ++f) {
          const int sl = rec_slot_of(info.z, f);
          if (sl < 0) continue;
          const int nb = nb_elem(a.nx, a.ny, e, f);
          if ((bits & (1u << (4 + f))) && it == 0) {
            const int pos = a.member_of[(size_t)d * a.E + nb] - first;
            if (pos >= mi) continue;  // not computed yet in the first sweep
          }
          y -= face_term<P, T, CG>(L::slot(r, rx, sl), a.out + ((size_t)d * a.E + nb) * N, f, i);
        }
        T* o = a.out + ((size_t)d * a.E + e) * N + i;
        if (it > 0) dmax = fmax(dmax, fabs(y - ldcg(o)));
        amax = fmax(amax, fabs(y));
        *o = y;
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

// Coupled group solved directly (groups within the direct limits).  The trace-system
// inverse T = (I + R)^{-1} of the group was formed by the factorisation; with it the
// group costs two passes over its member rows and one dense product:
//   z_a   = y_a - sum over faces of a fed from outside the group of W_{a,f} u_f
//   tau   = T (P z)          (P z: the members' z at the internal upwind face nodes)
//   psi_a = z_a - sum_{(a,f) internal} W_{a,f} tau_{a,f}
// Everything that does not depend on earlier levels (member info, y rows, the coupling
// list and, when small, T itself) is staged into shared memory ahead of the level.
template <int P, typename T>
struct GroupSmem {
  static constexpr int Q = P + 1, N = Q * Q, GM = group_direct_members(P);
  static constexpr int NC = kGroupMaxTrace / Q + 1;
  T z[GM * N];                                     // member rows: y, then z
  T rhs[kGroupMaxTrace];                           // P z
  T tau[kGroupMaxTrace];                           // trace unknowns
  T tinv[kGroupSmemTrace * kGroupSmemTrace];       // T (column-major) when nt <= kGroupSmemTrace
  uint4 info[GM];                                  // member record info
  uint32_t cpl[NC];                                // coupling: a | f << 8 | b << 16 | W slot << 24
  int cbase[GM + 1];                               // first coupling of each member
  int m, nt, gid;
};

template <int P, typename T>
__device__ __forceinline__ void group_stage(const SweepArgs<T>& a, int s0, GroupSmem<P, T>& g) {
  constexpr int Q = P + 1, N = Q * Q;
  using L = Rec<P, T>;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int first = a.slot_first[s0];
  const int cnt = a.slot_count[s0];           // <= group_direct_members(P) <= 32
  if (!(VEF_IN_RANGE(first, a.nmem, a.status) && VEF_IN_RANGE(first + cnt - 1, a.nmem, a.status))) return;
  const int gid = a.slot_gid[s0];
  uint4 info = make_uint4(0u, 0u, 0xffffffffu, 0u);
  uint32_t nbp = 0xffffffffu;
  if (lane < cnt) {
    info = *reinterpret_cast<const uint4*>(L::s_at(a.rec, first + lane));
    nbp = a.member_nbpos[first + lane];
    g.info[lane] = info;
  }
  // couplings of this member (faces inflow somewhere and shared with another member),
  // numbered by member then face: exclusive warp prefix sum of the counts
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
  for (int t = lane; t < cnt * N; t += 32) g.z[t] = ldcg(a.y + (size_t)(first + t / N) * L::kYStride + t % N);
  const int nt = total * Q;
  const T* Tg = a.grec + a.grp_toff[gid];
  if (nt <= kGroupSmemTrace)
    for (int t = lane; t < nt * nt; t += 32) g.tinv[t] = Tg[t];
  __syncwarp();
}

template <int P, typename T, bool CG = true>
__device__ __forceinline__ void group_solve_direct(const SweepArgs<T>& a, int d, int s0, GroupSmem<P, T>& g) {
  constexpr int Q = P + 1, N = Q * Q;
  using L = Rec<P, T>;
  const int lane = threadIdx.x & 31;
  const int first = a.slot_first[s0];
  if (!(VEF_IN_RANGE(first, a.nmem, a.status) && VEF_IN_RANGE(first + a.slot_count[s0] - 1, a.nmem, a.status)))
    return;
  const int m = g.m, nt = g.nt;
  // z: y minus the couplings to elements outside the group (earlier levels)
  for (int idx = lane; idx < m * N; idx += 32) {
    const int mi = idx / N, i = idx % N;
    const uint4 info = g.info[mi];
    const char* r = L::s_at(a.rec, first + mi);
    const char* rx = L::x_at(a.recx, first + mi);
    T z = g.z[idx];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int sl = rec_slot_of(info.z, f);
      if (sl < 0 || ((info.y >> (4 + f)) & 1u)) continue;
      const int nb = nb_elem(a.nx, a.ny, (int)info.x, f);
      z -= face_term<P, T, CG>(L::slot(r, rx, sl), a.out + ((size_t)d * a.E + nb) * N, f, i);
    }
    g.z[idx] = z;
  }
  __syncwarp();
  for (int j = lane; j < nt; j += 32) {
    const uint32_t cp = g.cpl[j / Q];
    const int b = (int)((cp >> 16) & 0xffu), f = (int)((cp >> 8) & 0xffu);
    g.rhs[j] = g.z[b * N + face_dof<P>((f + 2) & 3, j % Q)];
  }
  __syncwarp();
  const T* Tm = nt <= kGroupSmemTrace ? g.tinv : a.grec + a.grp_toff[g.gid];
  for (int r = lane; r < nt; r += 32) {
    T acc0 = 0, acc1 = 0;
    int j = 0;
    for (; j + 1 < nt; j += 2) {
      acc0 += Tm[j * nt + r] * g.rhs[j];
      acc1 += Tm[(j + 1) * nt + r] * g.rhs[j + 1];
    }
    if (j < nt) acc0 += Tm[j * nt + r] * g.rhs[j];
    g.tau[r] = acc0 + acc1;
  }
  __syncwarp();
  for (int idx = lane; idx < m * N; idx += 32) {
    const int mi = idx / N, i = idx % N;
    const char* r = L::s_at(a.rec, first + mi);
    const char* rx = L::x_at(a.recx, first + mi);
    T psi = g.z[idx];
    for (int c = g.cbase[mi]; c < g.cbase[mi + 1]; ++c) {
      const T* W = L::slot(r, rx, (int)(g.cpl[c] >> 24));
#pragma unroll
      for (int t = 0; t < Q; ++t) psi -= W[t * N + i] * g.tau[c * Q + t];
    }
    a.out[((size_t)d * a.E + g.info[mi].x) * N + i] = psi;
  }
  __syncwarp();
}

// Per warp: the staged prefixes of its single-element tasks' records (info + W slots 0, 1)
// and their y rows, for kSweepRounds rounds of two levels, filled by bulk copies (TMA)
// whose completion is counted on one mbarrier per level buffer.
constexpr int kSweepRounds = 2;

template <int P, typename T>
struct SweepSmem {
  static constexpr int SPC = (32 / ((P + 1) * (P + 1))) > 0 ? (32 / ((P + 1) * (P + 1))) : 1;
  alignas(16) unsigned char rec[2][kSweepRounds][SPC][Rec<P, T>::kStaged];
  alignas(16) unsigned char y[2][kSweepRounds][SPC][Rec<P, T>::kYBytes];
  uint64_t bar[2];
};

// dynamic shared memory of a sweep CTA: one SweepSmem per warp, then one GroupSmem per
// group warp of the cluster (group warps are the cluster's last warps, all in its last CTA)
__host__ __device__ constexpr int sweep_group_warps(int cluster_warps) {
  return cluster_warps >= 16 ? cluster_warps / 16 : 1;
}
template <int P, typename T>
__host__ __device__ constexpr size_t sweep_smem_bytes(int cta_warps, int cluster_warps) {
  return sizeof(SweepSmem<P, T>) * (size_t)cta_warps +
         sizeof(GroupSmem<P, T>) * (size_t)sweep_group_warps(cluster_warps);
}

// Poll limits of the bounded waits.  A try-wait on an mbarrier phase that is not complete
// suspends the thread for ~3.9 us per poll on GB300 (vef_wait_selftest measures it), so a
// staging wait gives up after ~1 s; a flag poll with its 64 ns sleep takes ~0.26 us, so a
// band wait of the fused apply gives up after ~1.1 s.  The longest legitimate wait (a
// direction waiting for the fused apply to reach its band) lasts milliseconds.
constexpr uint32_t kStageWaitIters = 1u << 18;

// Warps [0, nws) of a cluster take the single-element tasks; the last ng warps take the
// coupled groups, so a group's inner iteration never delays a warp's singles and its
// static data is staged while the previous level finishes.
template <int P, typename T, int MODE>
__device__ __forceinline__ void sweep_direction(const SweepArgs<T>& a, int d, int cs) {
  constexpr int Q = P + 1, N = Q * Q;
  using L = Rec<P, T>;
  constexpr int SPC = SweepSmem<P, T>::SPC;
  extern __shared__ __align__(16) unsigned char sweep_smem[];
  const int lane = threadIdx.x & 31;
  SweepSmem<P, T>& sm = reinterpret_cast<SweepSmem<P, T>*>(sweep_smem)[threadIdx.x >> 5];
  const int nw = cs * (blockDim.x >> 5);
  const int gw = (blockIdx.x % cs) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int ng = sweep_group_warps(nw);
  const int nws = nw > ng ? nw - ng : nw;   // one-warp clusters do both kinds
  const bool singles = gw < nws;
  const bool groups = gw >= nws || nw == 1;
  const int gidx = nw == 1 ? 0 : gw - nws;
  GroupSmem<P, T>* gsm = reinterpret_cast<GroupSmem<P, T>*>(
      sweep_smem + sizeof(SweepSmem<P, T>) * (blockDim.x >> 5));
  GroupSmem<P, T>& gs = gsm[groups ? gidx : 0];
  auto direct = [&](int slot) { return a.slot_gid != nullptr && a.slot_gid[slot] >= 0; };
  const int k0 = a.dir_lev0[d], k1 = a.dir_lev0[d + 1];
  const int i = lane % N;
  const int s_lane = lane / N;              // task slot of this lane inside a round
  const int stride = nws * SPC;
  // task offset of this warp at level k: the warps' order rotates from level to level, so
  // the warps that take a level's extra round are not the ones that took the previous
  // level's (those finish their staging last and would start every level late)
  auto wbase = [&](int k) { return ((gw + (k - k0) * 17) % nws) * SPC; };
  const bool lane_ok = singles && lane < SPC * N;
  if (lane == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
  }
  __syncwarp();
  // level table window in registers: lane j holds the table entries of levels kb + j and
  // kb + 32 + j; a level's entries are read with a shuffle, so the tables never sit on
  // the per-level critical path
  constexpr unsigned FULL = 0xffffffffu;
  int kb = k0;
  int lb0, lg0, lm0, lb1, lg1, lm1;
  auto load_win = [&](int base, int& lb, int& lg, int& lm) {
    const int kk = base + lane;
    lb = kk <= k1 ? a.lev_begin[kk] : 0;
    lg = kk < k1 ? a.lev_gbegin[kk] : 0;
    lm = kk < k1 ? a.lev_mbegin[kk] : 0;
  };
  load_win(k0, lb0, lg0, lm0);
  load_win(k0 + 32, lb1, lg1, lm1);
  auto lev_b = [&](int kk) { const int j = kk - kb; return __shfl_sync(FULL, j < 32 ? lb0 : lb1, j & 31); };
  auto lev_g = [&](int kk) { const int j = kk - kb; return __shfl_sync(FULL, j < 32 ? lg0 : lg1, j & 31); };
  auto lev_m = [&](int kk) { const int j = kk - kb; return __shfl_sync(FULL, j < 32 ? lm0 : lm1, j & 31); };
  unsigned phase[2] = {0u, 0u};
  bool pending[2] = {false, false};
  // stage level k into buffer b: up to kSweepRounds rounds of SPC consecutive members
  auto stage_level = [&](int k, int b) {
    const int n = lev_g(k) - lev_b(k), mb = lev_m(k);
    unsigned bytes = 0;
    int cnt[kSweepRounds];
#pragma unroll
    for (int r = 0; r < kSweepRounds; ++r) {
      const int t0 = wbase(k) + r * stride;
      cnt[r] = singles ? max(0, min(SPC, n - t0)) : 0;
      bytes += (unsigned)cnt[r] * (L::kStaged + L::kYBytes);
    }
    pending[b] = bytes > 0;
    if (!bytes) return;
    __syncwarp();
    if (lane == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&sm.bar[b], bytes);
#pragma unroll
      for (int r = 0; r < kSweepRounds; ++r) {
        if (!cnt[r]) continue;
        const long long m0 = mb + wbase(k) + r * stride;
        bulk_g2s(sm.rec[b][r][0], L::s_at(a.rec, m0), (unsigned)cnt[r] * L::kStaged, &sm.bar[b]);
        bulk_g2s(sm.y[b][r][0], a.y + m0 * L::kYStride, (unsigned)cnt[r] * L::kYBytes, &sm.bar[b]);
      }
    }
  };
  // once a staging wait gave up, this warp's staged buffers are never read again (they may
  // not have been filled); it keeps walking the levels so every barrier is still reached
  bool failed = false;
  auto wait_level = [&](int b) {
    if (!pending[b]) return;
    const bool ok = mbar_wait_data(&sm.bar[b], phase[b], kStageWaitIters, a.status);
    if (!ok && lane == 0) atomicOr(a.status, kDevTimeout);
    failed = failed || __any_sync(0xffffffffu, !ok);
    phase[b] ^= 1u;
    pending[b] = false;
  };
  if (singles) {
    stage_level(k0, 0);
    if (k0 + 1 < k1) stage_level(k0 + 1, 1);
  }
  int staged = -1;   // group slot whose static data sits in gs
  if (groups) {
    const int g0 = lev_g(k0) + gidx;
    if (g0 < lev_b(k0 + 1) && direct(g0)) {
      group_stage<P, T>(a, g0, gs);
      staged = g0;
    }
  }
  for (int k = k0; k < k1; ++k) {
    const int b = (k - k0) & 1;
    if (k - kb >= 32) {   // advance the window; the new half is first read 32 levels on
      kb += 32;
      lb0 = lb1; lg0 = lg1; lm0 = lm1;
      load_win(kb + 32, lb1, lg1, lm1);
    }
    const int sb = lev_b(k), sg = lev_g(k), se = lev_b(k + 1);
    if (singles) {
      const int nsingle = sg - sb, mb = lev_m(k), wb = wbase(k);
      wait_level(b);
      // staged rounds: issue every upwind load first, then the FMAs
      T u[kSweepRounds][2][Q];
      bool has[kSweepRounds];
#pragma unroll
      for (int r = 0; r < kSweepRounds; ++r) {
        has[r] = !failed && lane_ok && wb + r * stride + s_lane < nsingle;
        if (!has[r]) continue;
        const uint4 info = *reinterpret_cast<const uint4*>(sm.rec[b][r][s_lane]);
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
          const unsigned f = (info.z >> (8 * sl)) & 0xffu;
          if (f == 0xffu) continue;
          const T* un = a.out + ((size_t)d * a.E + nb_elem(a.nx, a.ny, (int)info.x, (int)f)) * N;
#pragma unroll
          for (int t = 0; t < Q; ++t) u[r][sl][t] = ldcg(un + face_dof<P>(((int)f + 2) & 3, t));
        }
      }
#pragma unroll
      for (int r = 0; r < kSweepRounds; ++r) {
        if (!has[r]) continue;
        const char* rs = (const char*)sm.rec[b][r][s_lane];
        const uint4 info = *reinterpret_cast<const uint4*>(rs);
        // two independent FMA chains (one per slot) joined by one add: 2(p+1) + 1 FP64
        // instructions on the critical path of the level
        T y0 = reinterpret_cast<const T*>(sm.y[b][r][s_lane])[i], y1 = 0;
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
          if (((info.z >> (8 * sl)) & 0xffu) == 0xffu) continue;
          const T* W = L::slot(rs, nullptr, sl);
#pragma unroll
          for (int t = 0; t < Q; ++t) {
            if (sl == 0) y0 = fma(-W[t * N + i], u[r][sl][t], y0);
            else y1 = fma(-W[t * N + i], u[r][sl][t], y1);
          }
        }
        T y = y0 + y1;
        if (((info.z >> 16) & 0xffu) != 0xffu) {   // rare: more than two interior inflow faces
          const char* rg = L::x_at(a.recx, mb + wb + r * stride + s_lane);
          for (int sl = 2; sl < 4; ++sl) {
            const unsigned f = (info.z >> (8 * sl)) & 0xffu;
            if (f == 0xffu) continue;
            y -= face_term<P, T>(L::slot(nullptr, rg, sl),
                                 a.out + ((size_t)d * a.E + nb_elem(a.nx, a.ny, (int)info.x, (int)f)) * N,
                                 (int)f, i);
          }
        }
        a.out[((size_t)d * a.E + info.x) * N + i] = y;
      }
      // rounds beyond the staged ones (levels wider than kSweepRounds * stride)
      for (int r = kSweepRounds; wb + r * stride < nsingle; ++r) {
        const int tl = wb + r * stride + s_lane;
        if (!failed && lane_ok && tl < nsingle) {
          const char* rg = L::s_at(a.rec, mb + tl);
          const char* rgx = L::x_at(a.recx, mb + tl);
          const uint4 info = *reinterpret_cast<const uint4*>(rg);
          T y = a.y[(size_t)(mb + tl) * L::kYStride + i];
          for (int sl = 0; sl < 4; ++sl) {
            const unsigned f = (info.z >> (8 * sl)) & 0xffu;
            if (f == 0xffu) continue;
            y -= face_term<P, T>(L::slot(rg, rgx, sl),
                                 a.out + ((size_t)d * a.E + nb_elem(a.nx, a.ny, (int)info.x, (int)f)) * N,
                                 (int)f, i);
          }
          a.out[((size_t)d * a.E + info.x) * N + i] = y;
        }
      }
    }
    if (groups) {
      for (int g = sg + gidx; g < se; g += ng) {
        if (direct(g)) {
          if (staged != g) group_stage<P, T>(a, g, gs);
          group_solve_direct<P, T>(a, d, g, gs);
        } else {
          group_solve<P, T, MODE>(a, d, g);
        }
        staged = -1;
      }
    }
    // publish this level; stage what later levels need while the barrier completes
    cluster_arrive();
    if (singles && k + 2 < k1) stage_level(k + 2, b);
    if (groups && k + 1 < k1) {
      const int g1 = lev_g(k + 1) + gidx;
      if (g1 < lev_b(k + 2) && direct(g1)) {
        group_stage<P, T>(a, g1, gs);
        staged = g1;
      }
    }
    cluster_wait();
  }
  // drain copies still in flight (none are issued for levels past the last one)
  wait_level(0);
  wait_level(1);
}

// one cluster per direction of one problem
template <int P, typename T, int MODE>
__global__ void __maxnreg__(128) sweep_kernel(SweepArgs<T> a) {
  sweep_direction<P, T, MODE>(a, blockIdx.x / a.cluster_size, a.cluster_size);
}

// batch of independent problems of one DG order: cluster c runs direction cmap[c].y of
// problem cmap[c].x, whose arguments sit in tab
template <int P, typename T, int MODE>
__global__ void __maxnreg__(128)
sweep_batch_kernel(const SweepArgs<T>* __restrict__ tab, const int2* __restrict__ cmap, int cluster_size) {
  const int2 pd = cmap[blockIdx.x / cluster_size];
  sweep_direction<P, T, MODE>(tab[pd.x], pd.y, cluster_size);   // the launch's cluster size
}

// ------------------------------------------------------------- single-CTA sweep
// One CTA of 16 warps per direction.  Warp 15 streams the records of the direction's
// single-element tasks (staged prefix, y row, trace slot ids) through a ring of chunk
// buffers with bulk copies, as far ahead as the ring allows (a bulk copy request costs
// ~150 issue cycles whatever its size, so a chunk holds several rounds of one level);
// warps 0..11 compute them, a round being 12 * SPC consecutive tasks of one level with
// one lane per dof row; warps
// 12..14 solve the level's coupled groups, one group per warp at a time, each staging its
// first group of the next level while the level finishes.  The upwind face values passed from one single-element task
// to a later one go through shared-memory trace slots whose ids the schedule assigned,
// so a level costs shared-memory latency and a named barrier over the 15 computing warps
// instead of an L2 round trip and a cluster barrier.  Other couplings (from group
// members, into a receiver's extra W slots, beyond the slot capacity) read the donor's
// psi from global memory, which every task writes.
template <int P, typename T>
struct CtaShape {
  static constexpr int Q = P + 1, N = Q * Q;
  using L = Rec<P, T>;
  static constexpr int kCompute = 12, kGroupWarps = 3, kProducer = 15, kThreads = 512;
  static constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  static constexpr int CH = kCompute * SPC;                     // tasks per round
  static constexpr int kTaskBytes = L::kStaged + L::kYBytes + 16;
  // rounds per chunk: about 48 KB of records per chunk
  static constexpr int RC = (48 * 1024) / (CH * kTaskBytes) > 8 ? 8
                          : ((48 * 1024) / (CH * kTaskBytes) < 1 ? 1 : (48 * 1024) / (CH * kTaskBytes));
  static constexpr int CK = RC * CH;                             // tasks per chunk
  // chunk buffer: CK staged record prefixes, CK y rows, CK slot-id quadruples
  static constexpr int kYOff = CK * L::kStaged;
  static constexpr int kTsOff = kYOff + CK * L::kYBytes;
  static constexpr int kRound = kTsOff + CK * 16;                // bytes of one chunk buffer
  static constexpr int kGroup = kGroupWarps * (((int)sizeof(GroupSmem<P, T>) + 15) / 16 * 16);
  static constexpr int kMaxRing = 16;
  static constexpr int kBars = 2 * kMaxRing * 8;
  static constexpr int kSmemMax = 227 * 1024;
  // bytes of shared memory for the trace slots when the ring keeps `rounds` buffers
  static constexpr int trace_budget(int rounds) { return kSmemMax - kGroup - kBars - rounds * kRound; }
};

// Fused apply: when the directions leave SMs free, the sweep launch is cooperative (every
// CTA resident) and its CTAs past the direction CTAs compute y = A^{-1} b band by band
// (kApplyBand levels of one direction, bands in order across the directions), publishing
// a release flag per band; a direction's producer and group warps acquire a band's flag
// before reading its y rows.  The workers wait for nothing, so the waits always end.
constexpr int kApplyBand = 8;
constexpr int kMinApplyCtas = 8;   // fewer free SMs: apply by a launch of its own
constexpr uint32_t kReadyWaitIters = 1u << 22;

template <int P, typename T, int MODE>
__device__ __forceinline__ void apply_worker(const SweepArgs<T>& a) {
  constexpr int N = (P + 1) * (P + 1);
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  const int w = (int)blockIdx.x - a.nd, nworkers = (int)gridDim.x - a.nd;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int total_levels = a.dir_lev0[a.nd];
  const long long units = (long long)a.bands * a.nd;
  for (long long u = w; u < units; u += nworkers) {
    const int band = (int)(u / a.nd), dd = (int)(u % a.nd);
    const int k0d = a.dir_lev0[dd], k1d = a.dir_lev0[dd + 1];
    const int ka = k0d + band * kApplyBand;
    if (ka >= k1d) continue;
    const int kz = min(k1d, ka + kApplyBand);
    const long long mb = a.lev_mbegin[ka];
    const long long me = kz < total_levels ? (long long)a.lev_mbegin[kz] : a.nmem;
    for (long long m0 = mb + (long long)warp * SPC; m0 < me; m0 += (long long)nw * SPC)
      apply_warp<P, T, MODE>(a, m0, me);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release_gpu(a.ready + (size_t)dd * a.bands + band, 1);
    }
  }
}

// One direction d of one problem in this CTA (the single-CTA sweep proper).
template <int P, typename T, int MODE>
__device__ __forceinline__ void sweep_cta_direction(const SweepArgs<T>& a, const int d) {
  using Sh = CtaShape<P, T>;
  using L = Rec<P, T>;
  constexpr int Q = P + 1, N = Q * Q, SPC = Sh::SPC, CH = Sh::CH, CK = Sh::CK;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char cta_smem[];
  constexpr int kGs = ((int)sizeof(GroupSmem<P, T>) + 15) / 16 * 16;
  uint64_t* full = reinterpret_cast<uint64_t*>(cta_smem + Sh::kGroup);
  uint64_t* empty = full + Sh::kMaxRing;
  T* tr = reinterpret_cast<T*>(cta_smem + Sh::kGroup + Sh::kBars);
  unsigned char* ring = cta_smem + Sh::kGroup + Sh::kBars + a.tr_bytes;
  const unsigned NB = (unsigned)a.ring;
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
  // level tables in a register window of 64 levels, read with shuffles
  int kb = k0;
  int lb0, lg0, lm0, lb1, lg1, lm1;
  auto load_win = [&](int base, int& lb, int& lg, int& lm) {
    const int kk = base + lane;
    lb = kk <= k1 ? a.lev_begin[kk] : 0;
    lg = kk < k1 ? a.lev_gbegin[kk] : 0;
    lm = kk < k1 ? a.lev_mbegin[kk] : 0;
  };
  load_win(k0, lb0, lg0, lm0);
  load_win(k0 + 32, lb1, lg1, lm1);
  auto lev_b = [&](int kk) { const int j = kk - kb; return __shfl_sync(FULL, j < 32 ? lb0 : lb1, j & 31); };
  auto lev_g = [&](int kk) { const int j = kk - kb; return __shfl_sync(FULL, j < 32 ? lg0 : lg1, j & 31); };
  auto lev_m = [&](int kk) { const int j = kk - kb; return __shfl_sync(FULL, j < 32 ? lm0 : lm1, j & 31); };
  auto advance = [&](int k) {
    if (k - kb >= 32) {
      kb += 32;
      lb0 = lb1; lg0 = lg1; lm0 = lm1;
      load_win(kb + 32, lb1, lg1, lm1);
    }
  };
  // producer waits (a buffer released, copies drained): they do not stop on the status bit,
  // the consumers always release and copies in flight must land before the CTA exits
  auto bounded_wait = [&](uint64_t* bar, unsigned parity) {
    uint32_t n = 0;
    while (!mbar_try_wait(bar, parity) && ++n < kStageWaitIters) {
    }
    if (n >= kStageWaitIters) atomicOr(a.status, kDevTimeout);
  };
  // consumer waits for a staged chunk: give up early on the status bit; a warp whose wait
  // gave up never reads a staged chunk again, but still releases every buffer and reaches
  // every level barrier
  bool failed = false;
  auto data_wait = [&](uint64_t* bar, unsigned parity) {
    const bool ok = mbar_wait_data(bar, parity, kStageWaitIters, a.status);
    if (!ok) atomicOr(a.status, kDevTimeout);
    failed = failed || __any_sync(0xffffffffu, !ok);
  };
  // ring position and phase parity of the next round
  auto next = [&](unsigned& b, unsigned& par) {
    if (++b == NB) { b = 0; par ^= 1u; }
  };
  // fused apply: wait (whole warp) until the y rows of level kk's band are written
  int ready_band = -1;
  auto wait_ready = [&](int kk) {
    if (a.ready == nullptr) return;
    const int band = (kk - k0) / kApplyBand;
    if (band <= ready_band) return;
    if (lane == 0) {
      const int* flag = a.ready + (size_t)d * a.bands + band;
      uint32_t n = 0;
      while (ld_acquire_gpu(flag) == 0 && ++n < kReadyWaitIters) {
        if (*(volatile unsigned int*)a.status & kDevTimeout) break;
        __nanosleep(64);
      }
      if (n >= kReadyWaitIters) atomicOr(a.status, kDevTimeout);
    }
    __syncwarp();
    ready_band = band;
  };

  if (warp == Sh::kProducer) {
    unsigned rc = 0, b = 0, par = 0;
    for (int k = k0; k < k1; ++k) {
      advance(k);
      const int nsingle = lev_g(k) - lev_b(k), mb = lev_m(k);
      if (nsingle > 0 && a.ready != nullptr) {
        wait_ready(k);
        if (lane == 0) fence_proxy_async_global();   // the y rows are read by bulk copies
      }
      for (int r0 = 0; r0 < nsingle; r0 += CK, ++rc, next(b, par)) {
        if (lane != 0) continue;
        if (rc >= NB) bounded_wait(&empty[b], par ^ 1u);   // the buffer's previous use was released
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
        bulk_g2s(rb + Sh::kYOff, a.y + m0 * L::kYStride, (unsigned)(cnt * L::kYBytes), &full[b]);
        bulk_g2s(rb + Sh::kTsOff, a.tslot + m0, (unsigned)(cnt * 16), &full[b]);
      }
    }
    // no copy may be in flight when the CTA exits (the consumers wait for every round;
    // this only matters after a timed-out wait)
    if (lane == 0)
      for (unsigned j = rc > NB ? rc - NB : 0u; j < rc; ++j) bounded_wait(&full[j % NB], (j / NB) & 1u);
    return;
  }

  const bool compute = warp < Sh::kCompute;
  const int i = lane % N, s_lane = lane / N;
  const int task = warp * SPC + s_lane;
  const bool lane_ok = compute && lane < SPC * N;
  // the faces dof row i lies on (two at a corner) and its node position on each; the
  // write slot of a face is 16-bit half `sh` of word y (faces 0, 1) or z (faces 2, 3)
  // of the task's slot ids; rows on no face get the sink id (no store)
  const int ia = i % Q, ib = i / Q;
  int fA = -1, pA = 0, fB = -1, pB = 0;
  auto on_face = [&](int f, int pos) {
    if (fA < 0) { fA = f; pA = pos; } else { fB = f; pB = pos; }
  };
  if (ib == 0) on_face(0, ia);
  if (ia == P) on_face(1, ib);
  if (ib == P) on_face(2, ia);
  if (ia == 0) on_face(3, ib);
  const bool zA = fA >= 2, zB = fB >= 2;
  const unsigned shA = 16u * (unsigned)(fA & 1), shB = 16u * (unsigned)(fB & 1);
  const unsigned keepA = fA >= 0 ? 0xffffu : 0u, keepB = fB >= 0 ? 0xffffu : 0u;
  const unsigned sinkA = fA >= 0 ? 0u : kTraceSink, sinkB = fB >= 0 ? 0u : kTraceSink;
  T* outd = a.out + (size_t)d * a.E * N;
  const int ntr = a.tr_bytes / (Q * (int)sizeof(T));   // trace slots in shared memory
  (void)ntr;
  if (threadIdx.x < Q) tr[kTraceZero * Q + threadIdx.x] = (T)0;
  auto direct = [&](int slot) { return a.slot_gid != nullptr && a.slot_gid[slot] >= 0; };
  const int gidx = warp - Sh::kCompute;   // group warp index (group warps only)
  GroupSmem<P, T>& gs = *reinterpret_cast<GroupSmem<P, T>*>(cta_smem + (compute ? 0 : gidx) * kGs);
  unsigned rb_i = 0, rpar = 0;
  int staged = -1;
  if (!compute) {
    const int g0 = lev_g(k0) + gidx;
    if (g0 < lev_b(k0 + 1) && direct(g0)) {
      wait_ready(k0);
      group_stage<P, T>(a, g0, gs);
      staged = g0;
    }
  }
  named_barrier(1, (Sh::kCompute + Sh::kGroupWarps) * 32);   // the zero trace is in place
  for (int k = k0; k < k1; ++k) {
    advance(k);
    const int sb = lev_b(k), sg = lev_g(k), se = lev_b(k + 1);
    if (compute) {
      const int nsingle = sg - sb, mb = lev_m(k);
      for (int c0 = 0; c0 < nsingle; c0 += CK) {
        const unsigned char* rb = ring + (size_t)rb_i * Sh::kRound;
        data_wait(&full[rb_i], rpar);
        const int cend = min(CK, nsingle - c0);
        for (int tk = task; tk - task < cend; tk += CH) {   // the chunk's rounds
          const int r0 = c0 + tk - task;
          if (!failed && lane_ok && tk < cend) {
            const char* rs = (const char*)rb + tk * L::kStaged;
            const uint4 info = *reinterpret_cast<const uint4*>(rs);
            const uint4 ts = *reinterpret_cast<const uint4*>(rb + Sh::kTsOff + tk * 16);
            if (!(VEF_IN_RANGE(info.x, a.E, a.status) && VEF_IN_RANGE(ts.x & 0xffffu, ntr, a.status) &&
                  VEF_IN_RANGE(ts.x >> 16, ntr, a.status)))
              continue;
            const T* W = L::slot(rs, nullptr, 0);   // slots 0, 1 back to back; absent ones are zero
            const T* u0 = tr + (ts.x & 0xffffu) * Q;
            const T* u1 = tr + (ts.x >> 16) * Q;
            T y = reinterpret_cast<const T*>(rb + Sh::kYOff + tk * L::kYBytes)[i];
            if constexpr (sizeof(T) == 8) {
              // FP64 issue is the limit: one chain of 2(p+1) FMAs
#pragma unroll
              for (int t = 0; t < Q; ++t) y = fma(-W[t * N + i], u0[t], y);
#pragma unroll
              for (int t = 0; t < Q; ++t) y = fma(-W[L::kSlot + t * N + i], u1[t], y);
            } else {
              // latency is the limit: two independent chains joined by one add
              T yb = 0;
#pragma unroll
              for (int t = 0; t < Q; ++t) {
                y = fma(-W[t * N + i], u0[t], y);
                yb = fma(-W[L::kSlot + t * N + i], u1[t], yb);
              }
              y += yb;
            }
            const int e = (int)info.x;
            if (ts.w & 1u) {   // rare: couplings read from global memory
#pragma unroll 1
              for (int sl = 0; sl < 4; ++sl) {
                const unsigned f = (info.z >> (8 * sl)) & 0xffu;
                if (f == 0xffu || (sl < 2 && ((ts.x >> (16 * sl)) & 0xffffu) != kTraceZero)) continue;
                const T* Ws = sl < 2 ? W + sl * L::kSlot
                                     : L::slot(nullptr, L::x_at(a.recx, (long long)mb + r0 + task), sl);
                const int nb = nb_elem(a.nx, a.ny, e, (int)f);
                if (!(VEF_IN_RANGE(nb, a.E, a.status) && VEF_IN_RANGE((long long)mb + r0 + task, a.nmem, a.status)))
                  continue;
                y -= face_term<P, T, false>(Ws, outd + (size_t)nb * N, (int)f, i);
              }
            }
            outd[(size_t)(e * N + i)] = y;
            // this row's face-node values for later single-element receivers (no store for
            // faces nobody reads: id kTraceSink)
            const unsigned idA = (((zA ? ts.z : ts.y) >> shA) & keepA) | sinkA;
            const unsigned idB = (((zB ? ts.z : ts.y) >> shB) & keepB) | sinkB;
            if (idA != kTraceSink && VEF_IN_RANGE(idA, ntr, a.status)) tr[idA * Q + pA] = y;
            if (idB != kTraceSink && VEF_IN_RANGE(idB, ntr, a.status)) tr[idB * Q + pB] = y;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[rb_i]);
        next(rb_i, rpar);
      }
    } else {
      if (sg + gidx < se) wait_ready(k);
      for (int g = sg + gidx; g < se; g += Sh::kGroupWarps) {
        if (direct(g)) {
          if (staged != g) group_stage<P, T>(a, g, gs);
          group_solve_direct<P, T, false>(a, d, g, gs);
        } else {
          group_solve<P, T, MODE, false>(a, d, g);
        }
        staged = -1;
      }
      if (k + 1 < k1) {
        const int g1 = lev_g(k + 1) + gidx, ge = lev_b(k + 2);
        if (g1 < ge && direct(g1)) {
          wait_ready(k + 1);
          group_stage<P, T>(a, g1, gs);
          staged = g1;
        }
        // the next level's group records (never staged by the producer) into L2: the
        // solves read their W slots twice
        for (int g = g1; g < ge; g += Sh::kGroupWarps) {
          const long long first = a.slot_first[g];
          const int cnt = a.slot_count[g];
          constexpr int kSL = (L::kStaged + 127) / 128, kXL = (L::kExtra + 127) / 128;
          for (int t = lane; t < cnt * (kSL + kXL); t += 32) {
            const int mi = t / (kSL + kXL), li = t % (kSL + kXL);
            prefetch_l2(li < kSL ? L::s_at(a.rec, first + mi) + li * 128
                                 : L::x_at(a.recx, first + mi) + (li - kSL) * 128);
          }
        }
      }
    }
    named_barrier(1, (Sh::kCompute + Sh::kGroupWarps) * 32);
  }
}

template <int P, typename T, int MODE>
__global__ void __maxnreg__(128) sweep_cta_kernel(SweepArgs<T> a) {
  if (a.ready != nullptr && (int)blockIdx.x >= a.nd) {
    apply_worker<P, T, MODE>(a);
    return;
  }
  sweep_cta_direction<P, T, MODE>(a, blockIdx.x);
}

// Batch of independent problems of one DG order: CTA c runs direction cmap[c].y of problem
// cmap[c].x, whose arguments (ring and trace-slot sizes included) sit in tab; the launch's
// dynamic shared memory covers the largest of them.
template <int P, typename T, int MODE>
__global__ void __maxnreg__(128)
sweep_cta_batch_kernel(const SweepArgs<T>* __restrict__ tab, const int2* __restrict__ cmap) {
  const int2 pd = cmap[blockIdx.x];
  sweep_cta_direction<P, T, MODE>(tab[pd.x], pd.y);
}

// -------------------------------------------------------------- FP64 residual (mixed)
// r = b - L psi for every (element, direction) in schedule order, one thread per dof row
// (the rows of consecutive tasks packed across the lanes: the kernel is bound by FP64
// issue, and n = 9 rows would leave 5 of 32 lanes idle), from the stored FP64 element
// matrix and inflow couplings; accumulates ||r||^2, ||b||^2.
template <int P>
__global__ void __launch_bounds__(128)
residual_kernel(long long nmem, long long E, int nx, int ny, long long nbf,
                const uint32_t* __restrict__ code, const uint16_t* __restrict__ finfo,
                const double* __restrict__ omega, const double* __restrict__ Mm,
                const double* __restrict__ nds, const double* __restrict__ bvol,
                const double* __restrict__ src_aniso, const double* __restrict__ inflow,
                const double* __restrict__ a64, const float* __restrict__ rec32,
                const double* __restrict__ psi, FaceTab<double> ft, double* __restrict__ r,
                double* __restrict__ norms) {
  constexpr int Q = P + 1, N = Q * Q, NQ = P + 2, B = N * N + 4 * Q * Q;
  const int lane = threadIdx.x & 31;
  double rr = 0.0, bb = 0.0;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < nmem * N; row += nthreads) {
  const long long m = row / N;
  const int i = (int)(row - m * N);
  {
    const uint32_t cd = code[m];
    const int d = (int)(cd >> 22), e = (int)(cd & 0x3fffffu);
    const uint16_t bits = finfo[(size_t)d * E + e];
    const double mu = omega[2 * d], eta = omega[2 * d + 1];
    const double* pe = psi + ((size_t)d * E + e) * N;
    const double* blk = a64 + m * (long long)B;
    const unsigned faces = reinterpret_cast<const uint4*>(Rec<P, float>::s_at(rec32, m))->z;
    double b = bvol[(size_t)e * N + i];
    if (src_aniso) {
      const double* Mr = Mm + ((size_t)e * N + i) * N;
      const double* qd = src_aniso + ((size_t)d * E + e) * N;
      for (int j = 0; j < N; ++j) b += Mr[j] * qd[j];
    }
    double Apsi = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) Apsi += blk[j * N + i] * pe[j];   // A column-major
    const int ia = i % Q, ib = i / Q;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      int pos = -1;
      if (f == 0 && ib == 0) pos = ia;
      if (f == 1 && ia == P) pos = ib;
      if (f == 2 && ib == P) pos = ia;
      if (f == 3 && ia == 0) pos = ib;
      if (pos < 0 || !(bits & (1u << f))) continue;
      const int nb = nb_elem(nx, ny, e, f);
      if (nb >= 0) {
        const int sl = rec_slot_of(faces, f);
        const double* C = blk + N * N + sl * Q * Q + pos * Q;
        const double* pn = psi + ((size_t)d * E + nb) * N;
#pragma unroll
        for (int t = 0; t < Q; ++t) Apsi += C[t] * pn[face_dof<P>((f + 2) & 3, t)];
      } else if (inflow) {
        const double* pb = inflow + ((size_t)d * nbf + bface(nx, ny, e, f)) * NQ;
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
          const double* v = nds + (((size_t)e * 4 + f) * NQ + k) * 2;
          const double sv = ft.w[k] * (mu * v[0] + eta * v[1]);
          if (sv < 0.0) b -= sv * pb[k] * ft.l[pos][k];
        }
      }
    }
    const double ri = b - Apsi;
    r[((size_t)d * E + e) * N + i] = ri;
    rr += ri * ri;
    bb += b * b;
  }
  }
  // block reduction, then one atomic pair per block
  __shared__ double red[2][32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, off);
    bb += __shfl_xor_sync(0xffffffffu, bb, off);
  }
  if (lane == 0) {
    red[0][threadIdx.x >> 5] = rr;
    red[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sr += red[0][w];
      sb += red[1][w];
    }
    atomicAdd(norms, sr);
    atomicAdd(norms + 1, sb);
  }
}

// Matrix-free form of the same residual, for a single transport inversion: nothing per
// (element, direction) is stored, the element operator is applied from the
// direction-independent M, Gx, Gy (A psi = sigma_t M psi - mu Gx psi - eta Gy psi) and the
// face terms at the face Gauss points,
//     sum_k c_k psi_hat(s_k) l_a(s_k),  c_k = w_k Omega.(n ds)_k,
// psi_hat = own trace where c_k >= 0, else the upwind neighbour's trace or psi_bar (the
// boundary data move to the right-hand side with the same sign, so they enter r alike).
// Per task this costs 3 n^2 FP64 FMAs for the volume part where the stored form costs
// n^2, but it skips the FP64 assembly (3 n^2 per task) and its n^2 + 4 (p+1)^2 stored
// words, so it is cheaper whenever the systems serve a single residual.
// Element-major: a CTA holds one element's M, Gx, Gy and normals in shared memory and walks
// its directions; a task spans N lanes (row i on lane i), 32 / N tasks per warp.  The face
// points (4 (p+2) per task) are spread over the task's lanes, their c_k psi_hat go through
// shared memory to the lanes of the face-node rows.  Grid-stride over the elements.
// With FY it also forms the correction sweep's y = A^{-1} r from the FP32 records (the
// apply pass, same arithmetic as apply_warp: r rounded to FP32, one FMA chain over j): the
// kernel is bound by its FP64 work, which hides the A^{-1} reads.
template <int P, bool FY>
__global__ void __launch_bounds__(128)
residual_mf_kernel(int D, long long E, int nx, int ny, long long nbf, const double* __restrict__ omega,
                   const double* __restrict__ sigma_t, const double* __restrict__ Mm,
                   const double* __restrict__ Gxm, const double* __restrict__ Gym,
                   const double* __restrict__ nds, const double* __restrict__ bvol,
                   const double* __restrict__ src_aniso, const double* __restrict__ inflow,
                   const double* __restrict__ psi, FaceTab<double> ft, double* __restrict__ r,
                   double* __restrict__ norms, const int* __restrict__ member_of,
                   const float* __restrict__ recx32, float* __restrict__ y32, long long nmem,
                   unsigned int* status) {
  constexpr int Q = P + 1, N = Q * Q, NQ = P + 2, LD = N + 1;
  constexpr int UPW = 32 / N, NPT = 4 * NQ, ROUNDS = (NPT + N - 1) / N;
  constexpr int GZ = NPT;                   // a zero block after the face points
  __shared__ double sM[N * LD], sX[N * LD], sY[N * LD];
  __shared__ double sN[4 * NQ * 2];
  __shared__ double sP[4][UPW][N];          // psi of each warp's tasks
  __shared__ double sG[4][UPW][NPT + NQ];   // c_k psi_hat at the face points, then zeros
  __shared__ double sB[4][UPW][NPT + NQ];   // c_k psi_bar at boundary inflow points (for ||b||)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int u = lane / N, li = lane % N;
  const int uc = u < UPW ? u : UPW - 1;
  // the faces row li lies on (two at a corner, none inside): offsets of their points in
  // sG (the zero block for a missing face) and the node position on each
  const int ia = li % Q, ib = li / Q;
  int oA = GZ, pA = 0, oB = GZ, pB = 0;
  {
    int nf = 0;
    auto on = [&](int f, int pos) {
      if (nf++ == 0) { oA = f * NQ; pA = pos; } else { oB = f * NQ; pB = pos; }
    };
    if (ib == 0) on(0, ia);
    if (ia == P) on(1, ib);
    if (ib == P) on(2, ia);
    if (ia == 0) on(3, ib);
  }
  double lA[NQ], lB[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    lA[k] = ft.l[pA][k];
    lB[k] = ft.l[pB][k];
  }
  if (u < UPW)
    for (int k = li; k < NQ; k += N) sG[warp][u][GZ + k] = sB[warp][u][GZ + k] = 0.0;
  double rr = 0.0, bb = 0.0;
  for (long long e = blockIdx.x; e < E; e += gridDim.x) {
    __syncthreads();   // the previous element's tables are no longer read
    for (int idx = tid; idx < N * N; idx += blockDim.x) {
      const int ra = idx / N, j = idx % N;
      const size_t g = (size_t)e * N * N + idx;
      sM[ra * LD + j] = Mm[g];
      sX[ra * LD + j] = Gxm[g];
      sY[ra * LD + j] = Gym[g];
    }
    for (int idx = tid; idx < 4 * NQ * 2; idx += blockDim.x) sN[idx] = nds[(size_t)e * 4 * NQ * 2 + idx];
    __syncthreads();
    const double st = sigma_t[e];
    const int ie = (int)(e % nx), je = (int)(e / nx);
    const bool on_boundary = ie == 0 || je == 0 || ie == nx - 1 || je == ny - 1;
    const double bv = bvol[(size_t)e * N + li];
    for (int d0 = warp * UPW; d0 < D; d0 += nwarps * UPW) {
      const int d = d0 + u;
      const bool valid = u < UPW && d < D;
      const int dd = valid ? d : 0;
      const double mu = omega[2 * dd], eta = omega[2 * dd + 1];
      const size_t rowbase = ((size_t)dd * E + e) * N;
      const double pi = valid ? psi[rowbase + li] : 0.0;
      __syncwarp();
      if (u < UPW) sP[warp][u][li] = pi;
      __syncwarp();
      // face points: c_k psi_hat, the trace taken from this element (c_k >= 0) or from the
      // upwind neighbour, one FMA chain either way; psi_bar where the face is the boundary
#pragma unroll
      for (int rd = 0; rd < ROUNDS; ++rd) {
        const int q = li + N * rd;
        if (u < UPW && q < NPT) {
          const int f = q / NQ, k = q % NQ;
          const double c = ft.w[k] * (mu * sN[(f * NQ + k) * 2] + eta * sN[(f * NQ + k) * 2 + 1]);
          const int nb = nb_elem(nx, ny, (int)e, f);
          const bool own = c >= 0.0;
          double tr = 0.0, tb = 0.0;
          if (own || nb >= 0) {
            const double* src = own ? &sP[warp][u][0] : psi + ((size_t)dd * E + nb) * N;
            const int fs = own ? f : ((f + 2) & 3);
#pragma unroll
            for (int t = 0; t < Q; ++t) tr = fma(ft.l[t][k], src[face_dof<P>(fs, t)], tr);
          } else if (inflow) {
            tr = tb = inflow[((size_t)dd * nbf + bface(nx, ny, (int)e, f)) * NQ + k];
          }
          sG[warp][u][q] = c * tr;
          sB[warp][u][q] = c * tb;
        }
      }
      // volume part, row li
      double am = 0.0, ax = 0.0, ay = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const double pj = sP[warp][uc][j];
        am = fma(sM[li * LD + j], pj, am);
        ax = fma(sX[li * LD + j], pj, ax);
        ay = fma(sY[li * LD + j], pj, ay);
      }
      double b = bv;
      if (src_aniso) {
        const double* qd = src_aniso + rowbase;
#pragma unroll
        for (int j = 0; j < N; ++j) b = fma(sM[li * LD + j], qd[j], b);
      }
      __syncwarp();
      double fs = 0.0, bs = 0.0;
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        fs = fma(sG[warp][uc][oA + k], lA[k], fs);
        fs = fma(sG[warp][uc][oB + k], lB[k], fs);
      }
      if (on_boundary && inflow) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
          bs = fma(sB[warp][uc][oA + k], lA[k], bs);
          bs = fma(sB[warp][uc][oB + k], lB[k], bs);
        }
      }
      const double ri = b - (st * am - mu * ax - eta * ay) - fs;
      if (valid) {
        r[rowbase + li] = ri;
        rr = fma(ri, ri, rr);
        bb = fma(b - bs, b - bs, bb);
      }
      if constexpr (FY) {
        using L = Rec<P, float>;
        const long long m = valid ? (long long)member_of[(size_t)dd * E + e] : 0;
        const bool ok = valid && VEF_IN_RANGE(m, nmem, status);
        const float rf = ok ? (float)ri : 0.0f;
        const float* ai = L::ainv(L::x_at(recx32, ok ? m : 0));
        float y = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const float bj = __shfl_sync(0xffffffffu, rf, (uc * N + j) & 31);
          if (ok) y += ai[j * N + li] * bj;
        }
        if (ok) y32[(size_t)m * L::kYStride + li] = y;
      }
    }
  }
  __shared__ double red[2][32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, off);
    bb += __shfl_xor_sync(0xffffffffu, bb, off);
  }
  if (lane == 0) {
    red[0][warp] = rr;
    red[1][warp] = bb;
  }
  __syncthreads();
  if (tid == 0) {
    double sr = 0.0, sb = 0.0;
    for (int w = 0; w < nwarps; ++w) {
      sr += red[0][w];
      sb += red[1][w];
    }
    atomicAdd(norms, sr);
    atomicAdd(norms + 1, sb);
  }
}

__global__ void cast_add_kernel(long long n, const float* __restrict__ delta, double* __restrict__ psi,
                                int accumulate) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  psi[t] = accumulate ? psi[t] + (double)delta[t] : (double)delta[t];
}

// phi[e][i] = sum_d w_d psi[d][e][i]
__global__ void phi_kernel(int D, long long En, const double* __restrict__ w,
                           const double* __restrict__ psi, double* __restrict__ phi) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= En) return;
  double s = 0.0;
  for (int d = 0; d < D; ++d) s += w[d] * psi[(size_t)d * En + t];
  phi[t] = s;
}

// out = max |a - b| (non-negative doubles order like their bit patterns)
__global__ void maxdiff_kernel(long long n, const double* __restrict__ a, const double* __restrict__ b,
                               unsigned long long* out) {
  double m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[t] - (b ? b[t] : 0.0)));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// ------------------------------------------------------------------------ host side
static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

struct SweepCall {
  Mesh* mesh;
  Schedule* S;
  const double* sigma_t;
  const double* sigma_s;
  const double* src_aniso;
  const double* inflow;
  cudaStream_t stream;
  double tol;
  int max_passes;
  int precision;
  int cluster_size;  // CTAs per direction cluster
  int cta_warps;     // warps per CTA
  bool group_iterative;  // solve every coupled group by the inner iteration
  bool cluster;      // cluster sweep kernel instead of the single-CTA one
  bool apply_separate;   // y = A^{-1} b by its own launch even when SMs are free
  bool fixed_passes;     // mixed: exactly max_passes sweeps, no residual of the last one
  bool residual_stored;  // mixed: residual from stored FP64 element systems (else matrix-free)
  int force_pivot;       // refactorise every task with partial pivoting (tests of the fallback)
  bool reuse_factors;    // keep the schedule's factorisation from the previous call
  bool fuse_rhs;         // single inversion: the factorisation also forms y = A^{-1} b
  bool y_ready;          // y of the current right-hand side is in place: no apply pass
};

// Host-side arguments of one problem's sweep (also the batch table entries).
template <int P, typename T>
static vef_status make_sweep_args(const SweepCall& c, const double* rhs, T* out, SweepArgs<T>& a) {
  Mesh& M = *c.mesh;
  Schedule& S = *c.S;
  a = SweepArgs<T>{};
  a.dir_lev0 = S.dir_lev0;
  a.lev_begin = S.lev_begin;
  a.lev_gbegin = S.lev_gbegin;
  a.lev_mbegin = S.lev_mbegin;
  a.member_info = S.member_info;
  a.member_nbpos = S.member_nbpos;
  a.slot_first = S.slot_first;
  a.slot_count = S.slot_count;
  const void* grec = std::is_same<T, double>::value ? S.grec64 : S.grec32;
  if (!c.group_iterative && S.ngroups > 0 && grec) {
    a.slot_gid = S.slot_gid;
    a.grp_toff = S.grp_toff;
    a.grec = (const T*)grec;
  }
  a.code = S.member_code;
  a.member_of = S.member_of;
  a.finfo = S.faceinfo;
  a.omega = S.omega_dev;
  a.rec = (const T*)(std::is_same<T, double>::value ? S.rec64 : S.rec32);
  a.recx = (const T*)((const char*)a.rec + S.members * (long long)Rec<P, T>::kStaged);
  a.bvol = M.bvol;
  a.src_aniso = c.src_aniso;
  a.Mm = M.Mmat;
  a.inflow = c.inflow;
  a.nds = (const T*)(std::is_same<T, double>::value ? (const void*)M.nds : (const void*)M.nds32);
  a.rhs = rhs;
  a.out = out;
  vef_status st = ensure_buffer(&M.ybuf, &M.ybuf_cap, (size_t)S.members * Rec<P, T>::kYBytes);
  if (st != VEF_OK) return st;
  a.y = (T*)M.ybuf;
  a.status = M.dev_status;
  a.nx = M.nx;
  a.ny = M.ny;
  a.E = M.E;
  a.nbf = M.nbf;
  a.nmem = S.members;
  const double eps = std::is_same<T, double>::value ? 2.2e-16 : 1.2e-7;
  a.tol = (T)std::max(c.tol, 8.0 * eps);
  a.max_inner = std::max(2, 4 * c.max_passes);
  a.ft = make_facetab<T>(M.tab);
  a.cluster_size = c.cluster_size;
  return VEF_OK;
}

template <int P, typename T, int MODE>
static vef_status launch_apply(const SweepCall& c, const SweepArgs<T>& a) {
  constexpr int N = (P + 1) * (P + 1);
  constexpr int SPC = (32 / N) > 0 ? (32 / N) : 1;
  KTimer kt(c.mesh, VEF_K_SOURCE, c.stream);
  const long long warps = (c.S->members + SPC - 1) / SPC;
  apply_kernel<P, T, MODE><<<nblk(warps * 32, 128), 128, 0, c.stream>>>(a, c.S->members);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}

// cluster launch configuration of the sweep kernels (clusters x cs CTAs of warps x 32)
template <int P, typename T, typename K>
static vef_status cluster_config(K kernel, long long clusters, int cs, int warps, cudaStream_t stream,
                                 cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3((unsigned)(clusters * cs));
  cfg.blockDim = dim3((unsigned)(32 * warps));
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.dynamicSmemBytes = sweep_smem_bytes<P, T>(warps, cs * warps);
  VEF_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)cfg.dynamicSmemBytes));
  if (cs > 8) VEF_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  return VEF_OK;
}

// Cluster shape of a sweep when the caller gives none: 8-warp CTAs and the largest
// cluster (at most 8 CTAs, the portable limit) for which the occupancy calculator
// reports room for all D direction clusters at once.  Directions never wait on each
// other, but a cluster that does not fit starts only when another has finished, which
// doubles the critical path.
template <int P, typename T, int MODE>
static vef_status auto_tile(int D, int& cs_out, int& warps_out) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;   // (device, D) -> CTAs per cluster
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  warps_out = 8;
  auto it = cache.find({dev, D});
  if (it != cache.end()) { cs_out = it->second; return VEF_OK; }
  int best = 1;
  for (int cs = 8; cs >= 1; --cs) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    vef_status st = cluster_config<P, T>(sweep_kernel<P, T, MODE>, 1, cs, warps_out, nullptr, cfg, attr);
    if (st != VEF_OK) return st;
    int fit = 0;
    VEF_CUDA_TRY(cudaOccupancyMaxActiveClusters(&fit, sweep_kernel<P, T, MODE>, &cfg));
    if (fit >= D) { best = cs; break; }
  }
  cache[{dev, D}] = best;
  cs_out = best;
  return VEF_OK;
}

// Single-CTA sweep: one 16-warp CTA per direction; the trace slots take what the schedule
// needs and the ring of round buffers the rest of the shared memory (at most 16 rounds).
template <int P, typename T, int MODE>
static vef_status launch_sweep_cta(const SweepCall& c, SweepArgs<T>& a) {
  using Sh = CtaShape<P, T>;
  const Schedule& S = *c.S;
  const int tr = (S.trace_slots * (P + 1) * (int)sizeof(T) + 15) / 16 * 16;
  const int rounds = std::min(Sh::kMaxRing, (Sh::trace_budget(0) - tr) / Sh::kRound);
  if (rounds < 2) {
    set_last_error("internal error: single-CTA sweep ring does not fit in shared memory");
    return VEF_ERR_INVALID_ARG;
  }
  a.tslot = S.tslot;
  a.ring = rounds;
  a.tr_bytes = tr;
  const size_t smem = (size_t)Sh::kGroup + Sh::kBars + tr + (size_t)rounds * Sh::kRound;
  auto kern = sweep_cta_kernel<P, T, MODE>;
  VEF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // the SMs the directions leave free apply A^{-1} inside the same (cooperative) launch
  int dev = 0, sms = 0, per_sm = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  VEF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  VEF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Sh::kThreads, smem));
  const int workers = per_sm * sms - S.D;
  cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
  VEF_CUDA_TRY(cudaStreamIsCapturing(c.stream, &capturing));
  // graph capture keeps the plain launch pair (no cooperative node in the graph); from p = 3
  // the apply's A^{-1} stream (n^2 words per task) is faster on every SM before the sweep
  // than on the SMs the directions leave free during it
  if (c.y_ready || c.apply_separate || P >= 3 || workers < kMinApplyCtas ||
      capturing != cudaStreamCaptureStatusNone) {
    if (!c.y_ready) {   // y already formed by the factorisation otherwise
      vef_status st = launch_apply<P, T, MODE>(c, a);
      if (st != VEF_OK) return st;
    }
    KTimer kt(c.mesh, VEF_K_SWEEP, c.stream);
    kern<<<(unsigned)S.D, Sh::kThreads, smem, c.stream>>>(a);
    VEF_CUDA_TRY(cudaGetLastError());
    return VEF_OK;
  }
  Mesh& M = *c.mesh;
  a.bands = (S.levels + kApplyBand - 1) / kApplyBand;
  a.nd = S.D;
  a.nmem = S.members;
  const size_t flag_bytes = (size_t)S.D * a.bands * sizeof(int);
  vef_status st = ensure_buffer((void**)&M.ready_flags, &M.ready_cap, flag_bytes);
  if (st != VEF_OK) return st;
  a.ready = M.ready_flags;
  VEF_CUDA_TRY(cudaMemsetAsync(M.ready_flags, 0, flag_bytes, c.stream));
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3((unsigned)(S.D + workers));
  cfg.blockDim = dim3(Sh::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.stream;
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  KTimer kt(c.mesh, VEF_K_SWEEP, c.stream);   // the sweep with its apply
  VEF_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a));
  return VEF_OK;
}

template <int P>
static int cta_capacity_p() {
  using Sh = CtaShape<P, double>;   // FP64 layout: the larger records, at least 3 rounds
  return std::max(0, std::min(0xfffe, Sh::trace_budget(3) / ((P + 1) * (int)sizeof(double))));
}

int cta_trace_capacity(int p) {
  switch (p) {
    case 1: return cta_capacity_p<1>();
    case 2: return cta_capacity_p<2>();
    case 3: return cta_capacity_p<3>();
    default: return cta_capacity_p<4>();
  }
}

template <int P, typename T, int MODE>
static vef_status launch_sweep(const SweepCall& c0, const double* rhs, T* out) {
  SweepCall c = c0;
  if (!c.cluster) {
    SweepArgs<T> a;
    vef_status st = make_sweep_args<P, T>(c, rhs, out, a);
    if (st != VEF_OK) return st;
    return launch_sweep_cta<P, T, MODE>(c, a);
  }
  if (c.cluster_size == 0) {
    vef_status st = auto_tile<P, T, MODE>(c.S->D, c.cluster_size, c.cta_warps);
    if (st != VEF_OK) return st;
  }
  SweepArgs<T> a;
  vef_status st = make_sweep_args<P, T>(c, rhs, out, a);
  if (st != VEF_OK) return st;
  if (!c.y_ready && (st = launch_apply<P, T, MODE>(c, a)) != VEF_OK) return st;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  if ((st = cluster_config<P, T>(sweep_kernel<P, T, MODE>, c.S->D, c.cluster_size, c.cta_warps, c.stream,
                                 cfg, attr)) != VEF_OK)
    return st;
  KTimer kt(c.mesh, VEF_K_SWEEP, c.stream);
  VEF_CUDA_TRY(cudaLaunchKernelEx(&cfg, sweep_kernel<P, T, MODE>, a));
  return VEF_OK;
}

// The FP64 residual of the mixed defect correction.  With form_y (matrix-free form only) it
// also writes the FP32 correction sweep's y = A^{-1} r, so that sweep skips its apply.
template <int P>
static vef_status launch_residual(const SweepCall& c, const double* psi, double* r, double* norms,
                                  bool form_y = false) {
  Mesh& M = *c.mesh;
  Schedule& S = *c.S;
  constexpr int N = (P + 1) * (P + 1);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  VEF_CUDA_TRY(cudaMemsetAsync(norms, 0, 2 * sizeof(double), c.stream));
  if (!c.residual_stored) {
    const float* recx32 = nullptr;
    float* y32 = nullptr;
    if (form_y) {
      vef_status st = ensure_buffer(&M.ybuf, &M.ybuf_cap, (size_t)S.members * Rec<P, float>::kYBytes);
      if (st != VEF_OK) return st;
      recx32 = (const float*)((const char*)S.rec32 + S.members * (long long)Rec<P, float>::kStaged);
      y32 = (float*)M.ybuf;
    }
    const unsigned egrid = (unsigned)std::min<long long>(M.E, (long long)sms * 16);
    KTimer kt(&M, VEF_K_RESIDUAL, c.stream);
    auto kern = residual_mf_kernel<P, false>;
    if constexpr (P == 3) {   // the only order whose correction sweeps take y from here
      if (form_y) kern = residual_mf_kernel<P, true>;
    }
    kern<<<egrid, 128, 0, c.stream>>>(
        S.D, M.E, M.nx, M.ny, M.nbf, S.omega_dev, c.sigma_t, M.Mmat, M.Gx, M.Gy, M.nds, M.bvol,
        c.src_aniso, c.inflow, psi, make_facetab<double>(M.tab), r, norms, S.member_of, recx32, y32,
        S.members, M.dev_status);
    VEF_CUDA_TRY(cudaGetLastError());
    return VEF_OK;
  }
  const unsigned grid = (unsigned)std::min<long long>(nblk(S.members * N, 128), (long long)sms * 16);
  KTimer kt(&M, VEF_K_RESIDUAL, c.stream);
  residual_kernel<P><<<grid, 128, 0, c.stream>>>(
      S.members, M.E, M.nx, M.ny, M.nbf, S.member_code, S.faceinfo, S.omega_dev, M.Mmat, M.nds,
      M.bvol, c.src_aniso, c.inflow, (const double*)S.a64, (const float*)S.rec32, psi,
      make_facetab<double>(M.tab), r, norms);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}

// One full transport inversion into psi (FP64 output), factors assumed current.
template <int P>
static vef_status solve_p(const SweepCall& c, double* psi, vef_info* info) {
  Mesh& M = *c.mesh;
  Schedule& S = *c.S;
  if (c.precision == VEF_FP64) {
    vef_status st = launch_sweep<P, double, 0>(c, nullptr, psi);
    if (info) { info->passes = 1; info->rel_residual = -1.0; }
    return st;
  }
  // mixed: FP32 sweeps inside FP64 defect correction
  const long long tot = (long long)S.D * M.E * M.n;
  size_t need = (size_t)tot * sizeof(double) + 64;
  vef_status st = ensure_buffer((void**)&M.work2, &M.work2_cap, need + (size_t)tot * sizeof(float));
  if (st != VEF_OK) return st;
  double* r = M.work2;
  double* norms = (double*)((char*)M.work2 + (size_t)tot * sizeof(double));
  float* delta = (float*)((char*)M.work2 + need);
  if ((st = launch_sweep<P, float, 0>(c, nullptr, delta)) != VEF_OK) return st;
  {
    KTimer kt(&M, VEF_K_SOURCE, c.stream);
    cast_add_kernel<<<nblk(tot, 256), 256, 0, c.stream>>>(tot, delta, psi, 0);
  }
  // correction sweeps apply A^{-1} to the residual themselves, except at p = 3 (where the
  // apply is a pass of its own) in the matrix-free form: there the residual kernel forms y
  const bool y_in_residual = P == 3 && !c.residual_stored && S.rec32 != nullptr;
  SweepCall cc = c;
  cc.y_ready = y_in_residual;
  int passes = 1;
  double rel = -1.0;
  for (int pass = 0; pass < c.max_passes; ++pass) {
    // fixed passes: the last sweep's residual is not formed, and nothing is read back
    if (c.fixed_passes && pass == c.max_passes - 1) break;
    if ((st = launch_residual<P>(c, psi, r, norms, y_in_residual)) != VEF_OK) return st;
    if (!c.fixed_passes) {
      double h[2];
      VEF_CUDA_TRY(cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
      VEF_CUDA_TRY(cudaStreamSynchronize(c.stream));
      rel = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
      if (rel <= c.tol) break;
    }
    if (!c.fixed_passes && pass == c.max_passes - 1) {
      unsigned int bit = kDevNotConverged;
      VEF_CUDA_TRY(cudaMemcpyAsync(M.dev_status + 4, &bit, sizeof(bit), cudaMemcpyHostToDevice, c.stream));
      break;
    }
    if ((st = launch_sweep<P, float, 1>(cc, r, delta)) != VEF_OK) return st;
    {
      KTimer kt(&M, VEF_K_SOURCE, c.stream);
      cast_add_kernel<<<nblk(tot, 256), 256, 0, c.stream>>>(tot, delta, psi, 1);
    }
    ++passes;
  }
  if (info && c.fixed_passes && passes > 1) {
    // the residual of the iterate the last correction started from
    double h[2];
    VEF_CUDA_TRY(cudaMemcpyAsync(h, norms, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
    VEF_CUDA_TRY(cudaStreamSynchronize(c.stream));
    rel = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
  }
  if (info) { info->passes = passes; info->rel_residual = rel; }
  return VEF_OK;
}

static vef_status solve(const SweepCall& c, double* psi, vef_info* info) {
  switch (c.mesh->p) {
    case 1: return solve_p<1>(c, psi, info);
    case 2: return solve_p<2>(c, psi, info);
    case 3: return solve_p<3>(c, psi, info);
    default: return solve_p<4>(c, psi, info);
  }
}

// The local factorisation, unless the caller asked to keep the one the schedule holds for
// this precision (VEF_REUSE_FACTORS: sigma_t unchanged).  Any fresh factorisation may
// follow a change of sigma_t, so it leaves only what it has just formed marked as current.
// With c.fuse_rhs the factorisation also forms y = A^{-1} b for the current right-hand side
// (bvol computed before), and the first sweep that follows skips its apply (c.y_ready).
static vef_status factor(SweepCall& c) {
  c.y_ready = false;
  const unsigned need = c.precision == VEF_FP64 ? 1u : (2u | (c.residual_stored ? 4u : 0u));
  if (c.reuse_factors && (c.S->factored & need) == need) return VEF_OK;
  FactorRhs rhs;
  rhs.bvol = c.mesh->bvol;
  rhs.src_aniso = c.src_aniso;
  rhs.inflow = c.inflow;
  vef_status st = factor_records(c.mesh, c.S, c.sigma_t, c.precision, c.residual_stored, c.force_pivot,
                                 c.fuse_rhs ? &rhs : nullptr, c.stream);
  if (st == VEF_OK) {
    c.S->factored = need;
    c.y_ready = c.fuse_rhs;
  }
  return st;
}

static vef_status launch_bvol(Mesh& M, const double* sigma_s, const double* phi_in,
                              const double* q_iso, cudaStream_t stream) {
  size_t cap = 0;
  if (!M.bvol) {
    vef_status st = ensure_buffer((void**)&M.bvol, &cap, (size_t)M.E * M.n * sizeof(double));
    if (st != VEF_OK) return st;
  }
  KTimer kt(&M, VEF_K_SOURCE, stream);
  bvol_kernel<<<nblk(M.E * M.n, 256), 256, 0, stream>>>(M.E, M.n, M.Mmat, sigma_s, phi_in, q_iso, M.bvol);
  VEF_CUDA_TRY(cudaGetLastError());
  return VEF_OK;
}

// Read back and clear the device status; map to a vef_status.
vef_status collect_status(Mesh& M, cudaStream_t stream, vef_info* info) {
  unsigned int h[8];
  VEF_CUDA_TRY(cudaMemcpyAsync(h, M.dev_status, sizeof(h), cudaMemcpyDeviceToHost, stream));
  VEF_CUDA_TRY(cudaStreamSynchronize(stream));
  unsigned int zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  VEF_CUDA_TRY(cudaMemcpyAsync(M.dev_status, zero, sizeof(zero), cudaMemcpyHostToDevice, stream));
  VEF_CUDA_TRY(cudaStreamSynchronize(stream));
  const unsigned bits = h[0] | h[4];
  if (info) {
    info->timed_out = (bits & kDevTimeout) ? 1 : 0;
    info->max_inner_iterations = (int)h[2];
    info->pivoted_tasks = (long long)h[kStatusPivoted];
  }
  if (bits & kDevBounds) { set_last_error("bounds check: a kernel met an index outside its array"); return VEF_ERR_BOUNDS; }
  if (bits & kDevTimeout) { set_last_error("a sweep dependency wait ran out"); return VEF_ERR_TIMEOUT; }
  if (bits & kDevSingular) { set_last_error("singular local element system"); return VEF_ERR_NOT_CONVERGED; }
  if (bits & kDevNotConverged) { set_last_error("an iteration reached its cap"); return VEF_ERR_NOT_CONVERGED; }
  if (bits & kDevNonpositive) { set_last_error("non-positive closure denominator"); return VEF_ERR_NONPOSITIVE_DENOM; }
  return VEF_OK;
}

static vef_status check_common(vef_mesh mesh, const double* omega, const double* weights, int D,
                               const vef_opts* opts) {
  if (!mesh) { set_last_error("mesh is NULL"); return VEF_ERR_INVALID_ARG; }
  if (!omega || !weights) { set_last_error("omega and weights (host arrays) are required"); return VEF_ERR_INVALID_ARG; }
  if (D < 1 || D > kMaxD) { set_last_error("D must be in 1..1023"); return VEF_ERR_INVALID_ARG; }
  for (int d = 0; d < D; ++d) {
    if (!std::isfinite(omega[2 * d]) || !std::isfinite(omega[2 * d + 1]) || !std::isfinite(weights[d])) {
      set_last_error("omega / weights must be finite");
      return VEF_ERR_INVALID_ARG;
    }
  }
  if (opts && opts->precision != VEF_FP64 && opts->precision != VEF_MIXED) {
    set_last_error("opts->precision must be VEF_FP64 or VEF_MIXED");
    return VEF_ERR_INVALID_ARG;
  }
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != mesh->impl.device) { set_last_error("mesh belongs to another device"); return VEF_ERR_INVALID_ARG; }
  return VEF_OK;
}

static void fill_opts(const vef_opts* o, SweepCall& c) {
  c.precision = o ? o->precision : VEF_FP64;
  const double deftol = c.precision == VEF_FP64 ? 1e-15 : 1e-13;
  c.tol = (o && o->tol > 0.0) ? o->tol : deftol;
  c.fixed_passes = o && o->tol < 0.0 && c.precision == VEF_MIXED;
  c.max_passes = (o && o->max_passes > 0) ? o->max_passes : (c.fixed_passes ? 2 : 8);
  // tile_override = 100 * (CTAs per direction cluster) + (warps per CTA); 0 = automatic
  const int t = (o && o->tile_override > 0) ? o->tile_override : 0;
  c.cluster_size = t ? std::min(16, std::max(1, t / 100)) : 0;
  c.cta_warps = t ? std::min(16, std::max(1, t % 100)) : 0;
  c.group_iterative = o && (o->flags & VEF_GROUPS_ITERATIVE);
  c.cluster = t != 0 || (o && (o->flags & VEF_SWEEP_CLUSTER));
  c.apply_separate = o && (o->flags & VEF_APPLY_SEPARATE);
  c.force_pivot = (o && (o->flags & VEF_PIVOT_ALWAYS)) ? 1 : 0;
  c.reuse_factors = o && (o->flags & VEF_REUSE_FACTORS);
}

static void schedule_info(const Schedule& S, vef_info* info) {
  if (!info) return;
  info->coupled_groups = S.coupled_groups;
  info->lagged_face_points = S.lagged_points;
  info->levels = S.levels;
}

}  // namespace vef

using namespace vef;

extern "C" vef_status vef_sweep(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                                const double* phi_in, const double* source, int source_aniso,
                                const double* inflow, const double* omega, const double* weights,
                                int D, const vef_opts* opts, double* psi, vef_info* info,
                                void* stream) {
  vef_status st = check_common(mesh, omega, weights, D, opts);
  if (st != VEF_OK) return st;
  if (!sigma_t || !sigma_s || !psi) { set_last_error("sigma_t, sigma_s and psi are required"); return VEF_ERR_INVALID_ARG; }
  Mesh& M = mesh->impl;
  cudaStream_t s = (cudaStream_t)stream;
  Schedule* S = get_schedule(&M, omega, weights, D, s, &st);
  if (!S) return st;
  SweepCall c{};
  c.mesh = &M;
  c.S = S;
  c.sigma_t = sigma_t;
  c.sigma_s = sigma_s;
  c.src_aniso = source_aniso ? source : nullptr;
  c.inflow = inflow;
  c.stream = s;
  fill_opts(opts, c);
  c.fuse_rhs = !c.apply_separate;   // a single inversion: y = A^{-1} b formed with the factors
  if ((st = launch_bvol(M, sigma_s, phi_in, source_aniso ? nullptr : source, s)) != VEF_OK) return st;
  if ((st = factor(c)) != VEF_OK) return st;
  if ((st = solve(c, psi, info)) != VEF_OK) return st;
  if (info) {
    schedule_info(*S, info);
    return collect_status(M, s, info);
  }
  return VEF_OK;
}

extern "C" vef_status vef_source_iterate(vef_mesh mesh, const double* sigma_t, const double* sigma_s,
                                         const double* phi0, const double* source, int source_aniso,
                                         const double* inflow, const double* omega,
                                         const double* weights, int D, int K, const vef_opts* opts,
                                         double* phi_out, double* psi, double* dphi_inf,
                                         vef_info* info, void* stream) {
  vef_status st = check_common(mesh, omega, weights, D, opts);
  if (st != VEF_OK) return st;
  if (!sigma_t || !sigma_s || !psi || !phi_out || K < 1) {
    set_last_error("sigma_t, sigma_s, psi, phi_out are required and K >= 1");
    return VEF_ERR_INVALID_ARG;
  }
  Mesh& M = mesh->impl;
  cudaStream_t s = (cudaStream_t)stream;
  Schedule* S = get_schedule(&M, omega, weights, D, s, &st);
  if (!S) return st;
  SweepCall c{};
  c.mesh = &M;
  c.S = S;
  c.sigma_t = sigma_t;
  c.sigma_s = sigma_s;
  c.src_aniso = source_aniso ? source : nullptr;
  c.inflow = inflow;
  c.stream = s;
  fill_opts(opts, c);
  c.residual_stored = true;   // the FP64 systems serve the residuals of all K inversions
  const long long En = M.E * M.n;
  if ((st = ensure_buffer((void**)&M.work, &M.work_cap, (size_t)2 * En * sizeof(double))) != VEF_OK)
    return st;
  double* cur = M.work;
  double* nxt = M.work + En;
  if (phi0) VEF_CUDA_TRY(cudaMemcpyAsync(cur, phi0, En * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else VEF_CUDA_TRY(cudaMemsetAsync(cur, 0, En * sizeof(double), s));
  if ((st = factor(c)) != VEF_OK) return st;
  vef_info last{};
  int total_passes = 0;
  for (int k = 0; k < K; ++k) {
    if ((st = launch_bvol(M, sigma_s, cur, source_aniso ? nullptr : source, s)) != VEF_OK) return st;
    if ((st = solve(c, psi, info ? &last : nullptr)) != VEF_OK) return st;
    total_passes += info ? last.passes : 1;
    {
      KTimer kt(&M, VEF_K_SOURCE, s);
      phi_kernel<<<nblk(En, 256), 256, 0, s>>>(D, En, S->weights_dev, psi, nxt);
    }
    if (dphi_inf) {
      VEF_CUDA_TRY(cudaMemsetAsync(dphi_inf + k, 0, sizeof(double), s));
      KTimer kt(&M, VEF_K_SOURCE, s);
      maxdiff_kernel<<<std::min<long long>(nblk(En, 256), 1024), 256, 0, s>>>(
          En, nxt, cur, (unsigned long long*)(dphi_inf + k));
    }
    std::swap(cur, nxt);
  }
  VEF_CUDA_TRY(cudaMemcpyAsync(phi_out, cur, En * sizeof(double), cudaMemcpyDeviceToDevice, s));
  VEF_CUDA_TRY(cudaGetLastError());
  if (info) {
    *info = last;
    info->passes = total_passes;
    schedule_info(*S, info);
    return collect_status(M, s, info);
  }
  return VEF_OK;
}

extern "C" vef_status vef_mesh_sync(vef_mesh mesh, void* stream) {
  if (!mesh) { set_last_error("mesh is NULL"); return VEF_ERR_INVALID_ARG; }
  return collect_status(mesh->impl, (cudaStream_t)stream, nullptr);
}

namespace vef {
vef_status factor_fp64(Mesh* mesh, Schedule* S, const double* sigma_t, cudaStream_t stream) {
  SweepCall c{};
  c.mesh = mesh;
  c.S = S;
  c.sigma_t = sigma_t;
  c.stream = stream;
  c.precision = VEF_FP64;
  c.max_passes = 8;
  c.tol = 1e-15;
  return factor(c);
}
}  // namespace vef

// ------------------------------------------------------------------------- batches
// Many independent problems: per problem the dependency-free kernels (right-hand side,
// factorisation unless reused, apply) run as usual; the sweep of all problems of one DG
// order is one launch with a CTA (or, as tuned, a cluster) per (problem, direction).
namespace vef {

// sweep form of a batch class: kBatchCta = one CTA per (problem, direction); otherwise
// 100 x (CTAs per direction cluster) + (warps per CTA) of the cluster form
constexpr int kBatchCta = 1;

struct BatchClass {
  std::vector<int> probs;          // problem indices of this DG order, largest first
  int2* cmap = nullptr;            // [clusters] (position in probs, direction)
  long long clusters = 0;
  SweepArgs<double>* tab_dev = nullptr;
  SweepArgs<double>* tab_host = nullptr;   // pinned
  int tile = 0;                    // tuned form (0 = library default, the single-CTA form)
  bool tile_cached = false;        // tile came from the tuner cache (not timed again)
  size_t cta_smem = 0;             // dynamic shared memory of the single-CTA form (largest problem)
  std::string key;                 // tuner cache key: device and problems of this class
};

}  // namespace vef

struct vef_batch_s {
  int device = 0;
  std::vector<vef::Mesh*> meshes;
  std::vector<vef::Schedule*> scheds;
  vef::BatchClass cls[vef::kMaxP + 1];
  bool swept = false;
  // the pinned argument tables are copied to the device asynchronously; the host rewrites
  // them only once the copies of the previous call have been done (event recorded after
  // them, outside stream capture)
  cudaEvent_t tab_copied = nullptr;
  bool tab_pending = false;
  ~vef_batch_s() {
    for (auto& c : cls) {
      cudaFree(c.cmap);
      cudaFree(c.tab_dev);
      cudaFreeHost(c.tab_host);
    }
    if (tab_copied) cudaEventDestroy(tab_copied);
  }
};

namespace vef {

template <int P>
static vef_status batch_launch_class(vef_batch_s& B, BatchClass& C, int tile, cudaStream_t s) {
  if (tile == kBatchCta) {
    using Sh = CtaShape<P, double>;
    auto kern = sweep_cta_batch_kernel<P, double, 0>;
    VEF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C.cta_smem));
    KTimer kt(B.meshes[C.probs[0]], VEF_K_SWEEP, s);
    kern<<<(unsigned)C.clusters, Sh::kThreads, C.cta_smem, s>>>((const SweepArgs<double>*)C.tab_dev,
                                                               (const int2*)C.cmap);
    VEF_CUDA_TRY(cudaGetLastError());
    return VEF_OK;
  }
  const int cs = std::min(16, std::max(1, tile / 100)), warps = std::min(16, std::max(1, tile % 100));
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  vef_status st = cluster_config<P, double>(sweep_batch_kernel<P, double, 0>, C.clusters, cs, warps, s, cfg, attr);
  if (st != VEF_OK) return st;
  KTimer kt(B.meshes[C.probs[0]], VEF_K_SWEEP, s);
  VEF_CUDA_TRY(cudaLaunchKernelEx(&cfg, sweep_batch_kernel<P, double, 0>, (const SweepArgs<double>*)C.tab_dev,
                                  (const int2*)C.cmap, cs));
  return VEF_OK;
}

static vef_status batch_launch(vef_batch_s& B, int p, int tile, cudaStream_t s) {
  BatchClass& C = B.cls[p];
  switch (p) {
    case 1: return batch_launch_class<1>(B, C, tile, s);
    case 2: return batch_launch_class<2>(B, C, tile, s);
    case 3: return batch_launch_class<3>(B, C, tile, s);
    default: return batch_launch_class<4>(B, C, tile, s);
  }
}

// shared memory layout of one problem's single-CTA sweep: trace slots, then as many ring
// buffers as fit (at most CtaShape::kMaxRing)
template <int P>
static vef_status cta_layout(const Schedule& S, int& tr, int& rounds, size_t& smem) {
  using Sh = CtaShape<P, double>;
  tr = (S.trace_slots * (P + 1) * (int)sizeof(double) + 15) / 16 * 16;
  rounds = std::min(Sh::kMaxRing, (Sh::trace_budget(0) - tr) / Sh::kRound);
  if (rounds < 2) {
    set_last_error("internal error: single-CTA sweep ring does not fit in shared memory");
    return VEF_ERR_INVALID_ARG;
  }
  smem = (size_t)Sh::kGroup + Sh::kBars + tr + (size_t)rounds * Sh::kRound;
  return VEF_OK;
}

template <int P>
static vef_status batch_prepare(const SweepCall& c, double* psi, SweepArgs<double>& a) {
  vef_status st = make_sweep_args<P, double>(c, nullptr, psi, a);
  if (st != VEF_OK) return st;
  int tr = 0, rounds = 0;
  size_t smem = 0;
  if ((st = cta_layout<P>(*c.S, tr, rounds, smem)) != VEF_OK) return st;
  a.tslot = c.S->tslot;
  a.ring = rounds;
  a.tr_bytes = tr;
  a.ready = nullptr;   // no fused apply in batches: the apply runs just below
  return launch_apply<P, double, 0>(c, a);
}

template <int P>
static size_t batch_cta_smem(const vef_batch_s& B, const BatchClass& C, vef_status* st) {
  size_t most = 0;
  for (int k : C.probs) {
    int tr = 0, rounds = 0;
    size_t smem = 0;
    if ((*st = cta_layout<P>(*B.scheds[k], tr, rounds, smem)) != VEF_OK) return 0;
    most = std::max(most, smem);
  }
  return most;
}

// ---- tuner cache: lines "<key> <tile>" in the file VEF_TUNE_CACHE names
static std::string batch_class_key(const vef_batch_s& B, const BatchClass& C, int p) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  uint64_t h = 1469598103934665603ull;   // FNV-1a over the class's problems
  auto mix = [&](long long v) {
    for (int b = 0; b < 8; ++b) { h ^= (uint64_t)((v >> (8 * b)) & 0xff); h *= 1099511628211ull; }
  };
  mix(p);
  for (int k : C.probs) {
    const Mesh& M = *B.meshes[k];
    mix(M.nx); mix(M.ny); mix(M.m); mix(B.scheds[k]->D); mix(B.scheds[k]->levels);
  }
  std::string name(prop.name);
  for (char& ch : name) if (ch == ' ') ch = '_';
  char buf[64];
  snprintf(buf, sizeof(buf), "-sm%d-p%d-%016llx", prop.multiProcessorCount, p, (unsigned long long)h);
  return name + buf;
}

static int tune_cache_lookup(const std::string& key) {
  const char* path = std::getenv("VEF_TUNE_CACHE");
  if (!path || !*path) return 0;
  FILE* f = std::fopen(path, "r");
  if (!f) return 0;
  char k[256];
  int tile = 0, found = 0;
  while (std::fscanf(f, "%255s %d", k, &tile) == 2)
    if (key == k && (tile == kBatchCta || (tile >= 101 && tile <= 1616))) found = tile;
  std::fclose(f);
  return found;
}

static void tune_cache_store(const std::string& key, int tile) {
  const char* path = std::getenv("VEF_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d\n", key.c_str(), tile);
  std::fclose(f);
}

}  // namespace vef

extern "C" vef_status vef_batch_create(const vef_mesh* meshes, int nprob, const double* const* omega,
                                       const double* const* weights, const int* D, vef_batch* out) {
  if (!meshes || !omega || !weights || !D || !out || nprob < 1) {
    set_last_error("meshes, omega, weights, D, out are required and nprob >= 1");
    return VEF_ERR_INVALID_ARG;
  }
  *out = nullptr;
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  std::unique_ptr<vef_batch_s> B(new vef_batch_s());
  B->device = dev;
  for (int k = 0; k < nprob; ++k) {
    vef_status st = check_common(meshes[k], omega[k], weights[k], D[k], nullptr);
    if (st != VEF_OK) return st;
    for (int j = 0; j < k; ++j)
      if (meshes[j] == meshes[k]) {
        set_last_error("each problem of a batch needs its own mesh handle");
        return VEF_ERR_INVALID_ARG;
      }
    Mesh* M = &meshes[k]->impl;
    Schedule* S = get_schedule(M, omega[k], weights[k], D[k], 0, &st);
    if (!S) return st;
    B->meshes.push_back(M);
    B->scheds.push_back(S);
    B->cls[M->p].probs.push_back(k);
  }
  for (int p = 1; p <= kMaxP; ++p) {
    BatchClass& C = B->cls[p];
    if (C.probs.empty()) continue;
    // longest dependency chains first, so the short problems fill in behind them
    std::stable_sort(C.probs.begin(), C.probs.end(), [&](int x, int y) {
      const Schedule& a = *B->scheds[x];
      const Schedule& b = *B->scheds[y];
      return a.levels != b.levels ? a.levels > b.levels : a.members > b.members;
    });
    vef_status st = VEF_OK;
    switch (p) {
      case 1: C.cta_smem = batch_cta_smem<1>(*B, C, &st); break;
      case 2: C.cta_smem = batch_cta_smem<2>(*B, C, &st); break;
      case 3: C.cta_smem = batch_cta_smem<3>(*B, C, &st); break;
      default: C.cta_smem = batch_cta_smem<4>(*B, C, &st); break;
    }
    if (st != VEF_OK) return st;
    C.key = batch_class_key(*B, C, p);
    C.tile = tune_cache_lookup(C.key);
    C.tile_cached = C.tile != 0;
    std::vector<int2> cmap;
    for (size_t j = 0; j < C.probs.size(); ++j)
      for (int d = 0; d < B->scheds[C.probs[j]]->D; ++d) cmap.push_back(make_int2((int)j, d));
    C.clusters = (long long)cmap.size();
    VEF_CUDA_TRY(cudaMalloc(&C.cmap, cmap.size() * sizeof(int2)));
    VEF_CUDA_TRY(cudaMemcpy(C.cmap, cmap.data(), cmap.size() * sizeof(int2), cudaMemcpyHostToDevice));
    VEF_CUDA_TRY(cudaMalloc(&C.tab_dev, C.probs.size() * sizeof(SweepArgs<double>)));
    VEF_CUDA_TRY(cudaMallocHost(&C.tab_host, C.probs.size() * sizeof(SweepArgs<double>)));
  }
  *out = B.release();
  return VEF_OK;
}

extern "C" vef_status vef_batch_destroy(vef_batch batch) {
  if (!batch) return VEF_OK;
  cudaDeviceSynchronize();
  delete batch;
  return VEF_OK;
}

extern "C" vef_status vef_batch_sweep(vef_batch batch, const double* const* sigma_t,
                                      const double* const* sigma_s, const double* const* phi_in,
                                      const double* const* source, const double* const* inflow,
                                      double* const* psi, const vef_opts* opts, vef_info* info,
                                      void* stream) {
  if (!batch || !sigma_t || !sigma_s || !psi) {
    set_last_error("batch, sigma_t, sigma_s and psi are required");
    return VEF_ERR_INVALID_ARG;
  }
  if (opts && opts->precision != VEF_FP64) {
    set_last_error("batched sweeps run in FP64");
    return VEF_ERR_NOT_IMPLEMENTED;
  }
  int dev = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != batch->device) { set_last_error("batch belongs to another device"); return VEF_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  vef_batch_s& B = *batch;
  const int n = (int)B.meshes.size();
  for (int k = 0; k < n; ++k)
    if (!sigma_t[k] || !sigma_s[k] || !psi[k]) {
      set_last_error("sigma_t, sigma_s and psi entries are required for every problem");
      return VEF_ERR_INVALID_ARG;
    }
  cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
  VEF_CUDA_TRY(cudaStreamIsCapturing(s, &capturing));
  if (B.tab_pending && capturing == cudaStreamCaptureStatusNone) {
    // the previous call's table copies must have read the tables before they change
    VEF_CUDA_TRY(cudaEventSynchronize(B.tab_copied));
    B.tab_pending = false;
  }
  for (int p = 1; p <= kMaxP; ++p) {
    BatchClass& C = B.cls[p];
    for (size_t j = 0; j < C.probs.size(); ++j) {
      const int k = C.probs[j];
      SweepCall c{};
      c.mesh = B.meshes[k];
      c.S = B.scheds[k];
      c.sigma_t = sigma_t[k];
      c.sigma_s = sigma_s[k];
      c.src_aniso = nullptr;
      c.inflow = inflow ? inflow[k] : nullptr;
      c.stream = s;
      fill_opts(opts, c);
      vef_status st = launch_bvol(*c.mesh, sigma_s[k], phi_in ? phi_in[k] : nullptr,
                                  source ? source[k] : nullptr, s);
      if (st != VEF_OK) return st;
      if ((st = factor(c)) != VEF_OK) return st;
      switch (p) {
        case 1: st = batch_prepare<1>(c, psi[k], C.tab_host[j]); break;
        case 2: st = batch_prepare<2>(c, psi[k], C.tab_host[j]); break;
        case 3: st = batch_prepare<3>(c, psi[k], C.tab_host[j]); break;
        default: st = batch_prepare<4>(c, psi[k], C.tab_host[j]); break;
      }
      if (st != VEF_OK) return st;
    }
  }
  for (int p = 1; p <= kMaxP; ++p) {
    BatchClass& C = B.cls[p];
    if (C.probs.empty()) continue;
    VEF_CUDA_TRY(cudaMemcpyAsync(C.tab_dev, C.tab_host, C.probs.size() * sizeof(SweepArgs<double>),
                                 cudaMemcpyHostToDevice, s));
  }
  if (capturing == cudaStreamCaptureStatusNone) {
    if (!B.tab_copied) VEF_CUDA_TRY(cudaEventCreateWithFlags(&B.tab_copied, cudaEventDisableTiming));
    VEF_CUDA_TRY(cudaEventRecord(B.tab_copied, s));
    B.tab_pending = true;
  }
  for (int p = 1; p <= kMaxP; ++p) {
    BatchClass& C = B.cls[p];
    if (C.probs.empty()) continue;
    const int tile = (opts && opts->tile_override > 0) ? opts->tile_override : (C.tile ? C.tile : kBatchCta);
    vef_status st = batch_launch(B, p, tile, s);
    if (st != VEF_OK) return st;
  }
  B.swept = true;
  if (info) {
    info->passes = 1;
    info->rel_residual = -1.0;
    info->coupled_groups = 0;
    info->lagged_face_points = 0;
    info->levels = 0;
    info->max_inner_iterations = 0;
    info->timed_out = 0;
    vef_status worst = VEF_OK;
    for (int k = 0; k < n; ++k) {
      vef_info one{};
      vef_status st = collect_status(*B.meshes[k], s, &one);
      if (st != VEF_OK && worst == VEF_OK) worst = st;
      info->coupled_groups += B.scheds[k]->coupled_groups;
      info->lagged_face_points += B.scheds[k]->lagged_points;
      info->levels = std::max(info->levels, B.scheds[k]->levels);
      info->max_inner_iterations = std::max(info->max_inner_iterations, one.max_inner_iterations);
      info->timed_out |= one.timed_out;
    }
    return worst;
  }
  return VEF_OK;
}

extern "C" vef_status vef_batch_tune(vef_batch batch, void* stream, int* tiles_out) {
  if (!batch) { set_last_error("batch is NULL"); return VEF_ERR_INVALID_ARG; }
  if (!batch->swept) { set_last_error("call vef_batch_sweep once before tuning"); return VEF_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  static const int candidates[] = {kBatchCta, 204, 208, 404, 408, 804, 808, 1604};
  cudaEvent_t e0, e1;
  VEF_CUDA_TRY(cudaEventCreate(&e0));
  VEF_CUDA_TRY(cudaEventCreate(&e1));
  for (int p = 1; p <= kMaxP; ++p) {
    BatchClass& C = batch->cls[p];
    if (tiles_out) tiles_out[p - 1] = 0;
    if (C.probs.empty()) continue;
    if (C.tile_cached) {   // chosen by an earlier tuning of the same problems on this device
      if (tiles_out) tiles_out[p - 1] = C.tile;
      continue;
    }
    float best = 1e30f;
    int best_tile = kBatchCta;
    for (int tile : candidates) {
      vef_status st = batch_launch(*batch, p, tile, s);   // warm-up (also checks the shape launches)
      if (st != VEF_OK) {
        // a shape that cannot launch is skipped; an error left by the device is not
        const cudaError_t q = cudaStreamQuery(s);
        if (q != cudaSuccess && q != cudaErrorNotReady) return cuda_fail(q, "batch tuning launch");
        continue;
      }
      VEF_CUDA_TRY(cudaEventRecord(e0, s));
      for (int r = 0; r < 3; ++r)
        if ((st = batch_launch(*batch, p, tile, s)) != VEF_OK) break;
      VEF_CUDA_TRY(cudaEventRecord(e1, s));
      VEF_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      VEF_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (st == VEF_OK && ms < best) {
        best = ms;
        best_tile = tile;
      }
    }
    C.tile = best_tile;
    tune_cache_store(C.key, best_tile);
    if (tiles_out) tiles_out[p - 1] = best_tile;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return VEF_OK;
}
