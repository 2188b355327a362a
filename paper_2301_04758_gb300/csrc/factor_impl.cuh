// Local factorisation of the upwind element systems (template; included once per order) (no inter-element dependencies).
//
// For direction d and element e the element matrix is
//     A = sigma_t M - mu Gx - eta Gy + sum_f sum_k max(c_k, 0) l_a(s_k) l_b(s_k)
// (outflow face terms on the face nodes a, b; c_k = w_k Omega . (n ds)_k), and the
// coupling to the upwind neighbour across an inflow face f is
//     (Cin_f)_{a t} = sum_k min(c_k, 0) l_a(s_k) l_t(s_k),
// acting on the neighbour's face-node values.  One thread per (element, direction)
// assembles A, inverts it in place (Gauss-Jordan) and forms W_f = A^{-1} Cin_f for the
// interior inflow faces.  Record per (element, direction), in schedule order:
//     [element, face bits, slot faces][W slots, column-major n x (p+1)][A^{-1} column-major]
// (see Rec in device.cuh).
#pragma once
#include <algorithm>
#include <type_traits>

#include "device.cuh"

#ifndef VEF_FACTOR_P
#error "define VEF_FACTOR_P (1..4) before including factor_impl.cuh"
#endif

namespace vef {
namespace {

static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// products of the face Lagrange values at the face Gauss points, l_a(s_k) l_b(s_k)
template <typename T>
struct FaceLL {
  T ll[kMaxP + 1][kMaxP + 1][kMaxNq];
};

template <typename T>
inline FaceLL<T> make_facell(const Tab1D& t) {
  FaceLL<T> f{};
  for (int a = 0; a <= t.p; ++a)
    for (int b = 0; b <= t.p; ++b)
      for (int k = 0; k < t.nq; ++k) f.ll[a][b][k] = (T)(t.l[a][k] * t.l[b][k]);
  return f;
}

// ------------------------------------------------------------------- fused right-hand side
// For a single transport inversion the factorisation also forms y = A^{-1} b, with b the
// task's right-hand side entry as the sweep's own apply forms it (bvol, the anisotropic
// source's M q_d, minus the boundary inflow where the face point is inflow), so the sweep
// launch that follows needs no apply pass.  bvol == null: no y.
template <typename T>
struct RhsArgs {
  const double* bvol;       // [E][n]
  const double* src_aniso;  // [D][E][n] or null
  const double* inflow;     // [D][nbf][nq] or null
  const double* Mm64;       // FP64 mass matrices (anisotropic source)
  T* y;                     // y rows in schedule order, Rec<P, T>::kYStride apart
  long long nbf;
};

template <int P, typename T>
__device__ __forceinline__ T rhs_b(const RhsArgs<T>& r, const FaceTab<T>& ft, const T* __restrict__ nds,
                                   int nx, int ny, long long E, int d, int e, int j, uint16_t bits, T mu,
                                   T eta) {
  constexpr int Q = P + 1, N = Q * Q, NQ = P + 2;
  double b = r.bvol[(size_t)e * N + j];
  if (r.src_aniso) {
    const double* Mr = r.Mm64 + ((size_t)e * N + j) * N;
    const double* qd = r.src_aniso + ((size_t)d * E + e) * N;
#pragma unroll
    for (int jj = 0; jj < N; ++jj) b += Mr[jj] * qd[jj];
  }
  T bt = (T)b;
  if (r.inflow) {
    const int ia = j % Q, ib = j / Q;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!(bits & (1u << f))) continue;
      if (nb_elem(nx, ny, e, f) >= 0) continue;
      int pos = -1;
      if (f == 0 && ib == 0) pos = ia;
      if (f == 1 && ia == P) pos = ib;
      if (f == 2 && ib == P) pos = ia;
      if (f == 3 && ia == 0) pos = ib;
      if (pos < 0) continue;
      const double* pb = r.inflow + ((size_t)d * r.nbf + bface(nx, ny, e, f)) * NQ;
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        const T* v = nds + (((size_t)e * 4 + f) * NQ + k) * 2;
        const T sv = ft.w[k] * (mu * v[0] + eta * v[1]);
        if (sv < (T)0) bt -= sv * (T)pb[k] * ft.l[pos][k];
      }
    }
  }
  return bt;
}

// ------------------------------------------------------------------- pivot guard
// The element solves eliminate without pivoting.  A task whose pivot at some step falls
// below 2^VEF_PIVOT_FLOOR_LOG2_* times the largest entry of that row of the assembled
// matrix (or is zero, not finite, or above 2^1000) is appended to a list and refactorised
// with partial pivoting by factor_pivot_kernel, which overwrites its record.  Magnitudes
// are compared through the high word of their bit pattern with the sign cleared (exponent
// and leading mantissa bits), so the guard costs integer operations only.
template <typename T> struct PivotFloor;
template <> struct PivotFloor<double> {
  static __device__ __forceinline__ int mag(double x) { return __double2hiint(x) & 0x7fffffff; }
  static constexpr int kShift = (-VEF_PIVOT_FLOOR_LOG2_FP64) << 20;
  static constexpr int kHuge = (1000 + 1023) << 20;   // 2^1000: its reciprocal would flush
};
template <> struct PivotFloor<float> {
  static __device__ __forceinline__ int mag(float x) { return __float_as_int(x) & 0x7fffffff; }
  static constexpr int kShift = (-VEF_PIVOT_FLOOR_LOG2_FP32) << 23;
  static constexpr int kHuge = (120 + 127) << 23;      // 2^120
};
// pivot too small against the row scale (given as mag() of the row's largest entry), or
// too large for the reciprocal of pivot_rcp
template <typename T>
__device__ __forceinline__ bool small_pivot(T piv, int scale_mag) {
  return !(fabs(piv) > tiny_pivot<T>()) || PivotFloor<T>::mag(piv) < scale_mag - PivotFloor<T>::kShift ||
         PivotFloor<T>::mag(piv) >= PivotFloor<T>::kHuge;
}
__device__ __forceinline__ void pivot_list_append(unsigned int* count, unsigned int* list, long long m) {
  const unsigned idx = atomicAdd(count, 1u);
  list[idx] = (unsigned)m;   // at most one entry per task: the list holds every task
}

// ------------------------------------------------------------------- factorisation
// One (element, direction) task in one thread: assemble A and the inflow couplings,
// invert A in place by Gauss-Jordan (without pivoting and with the guard above, or with
// partial pivoting for the fallback), write the record.  Returns whether the guard fired.
template <int P, typename T, bool PIVOTED, bool Y>
__device__ __forceinline__ bool factor_task(long long m, long long nmem, const uint32_t* __restrict__ code,
                                            const uint16_t* __restrict__ finfo, const double* __restrict__ omega,
                                            const double* __restrict__ sigma_t, const T* __restrict__ Mm,
                                            const T* __restrict__ Gxm, const T* __restrict__ Gym,
                                            const T* __restrict__ nds, const FaceTab<T>& ft, const FaceLL<T>& fll,
                                            int nx, int ny, long long E, T* __restrict__ rec,
                                            unsigned int* status, const RhsArgs<T>& rhs) {
  constexpr int Q = P + 1, N = Q * Q, NQ = P + 2;
  using L = Rec<P, T>;
  const uint32_t c = code[m];
  const int d = (int)(c >> 22), e = (int)(c & 0x3fffffu);
  if (!VEF_IN_RANGE(e, E, status)) return false;
  const T mu = (T)omega[2 * d], eta = (T)omega[2 * d + 1];
  const T st = (T)sigma_t[e];
  const uint16_t bits = finfo[(size_t)d * E + e];
  T A[N * N];
  const T* Me = Mm + (size_t)e * N * N;
  const T* Xe = Gxm + (size_t)e * N * N;
  const T* Ye = Gym + (size_t)e * N * N;
#pragma unroll
  for (int ij = 0; ij < N * N; ++ij) A[ij] = st * Me[ij] - mu * Xe[ij] - eta * Ye[ij];
  // face terms: the outflow part only where some point is outflow, the inflow coupling
  // only for the faces that get a W slot (interior neighbour, some point inflow)
  T Cin[4][Q][Q];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    T cp[NQ], cm[NQ];
    bool anyout = false;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const T* v = nds + (((size_t)e * 4 + f) * NQ + k) * 2;
      const T s = ft.w[k] * (mu * v[0] + eta * v[1]);
      cp[k] = s > (T)0 ? s : (T)0;
      cm[k] = s < (T)0 ? s : (T)0;
      anyout = anyout || s > (T)0;
    }
    const bool need_in = (bits & (1u << f)) && nb_elem(nx, ny, e, f) >= 0;
    if (anyout) {
#pragma unroll
      for (int a = 0; a < Q; ++a)
#pragma unroll
        for (int b = 0; b < Q; ++b) {
          T vo = 0;
#pragma unroll
          for (int k = 0; k < NQ; ++k) vo = fma(cp[k], fll.ll[a][b][k], vo);
          A[face_dof<P>(f, a) * N + face_dof<P>(f, b)] += vo;
        }
    }
#pragma unroll
    for (int a = 0; a < Q; ++a)
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        T vi = 0;
        if (need_in) {
#pragma unroll
          for (int k = 0; k < NQ; ++k) vi = fma(cm[k], fll.ll[a][b][k], vi);
        }
        Cin[f][a][b] = vi;
      }
  }
  bool bad = false;
  if constexpr (!PIVOTED) {
    // in-place Gauss-Jordan inversion without pivoting: the upwind element matrices keep
    // their pivots well away from zero (a scan over the level-symmetric sets, p = 1..4,
    // void to optically thick and strongly curved elements finds the smallest pivot at
    // 0.1 of its row's largest entry); the guard hands any other task to the fallback
    int scl[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      int mx = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) mx = max(mx, PivotFloor<T>::mag(A[i * N + j]));
      scl[i] = mx;
    }
    constexpr int KU = P <= 2 ? N : 1;
#pragma unroll KU
    for (int k = 0; k < N; ++k) {
      const T piv = A[k * N + k];
      bad = bad || small_pivot<T>(piv, scl[k]);
      const T inv = pivot_rcp(piv);
#pragma unroll
      for (int j = 0; j < N; ++j)
        if (j != k) A[k * N + j] *= inv;
      A[k * N + k] = inv;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        if (i == k) continue;
        const T fct = A[i * N + k];
#pragma unroll
        for (int j = 0; j < N; ++j)
          if (j != k) A[i * N + j] -= fct * A[k * N + j];
        A[i * N + k] = -fct * inv;
      }
    }
  } else {
    // Gauss-Jordan with partial pivoting: rows interchanged at each step, the
    // interchanges undone as column interchanges (last first) at the end
    int perm[N];
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      int r = k;
      T best = fabs(A[k * N + k]);
#pragma unroll 1
      for (int i = k + 1; i < N; ++i)
        if (fabs(A[i * N + k]) > best) { best = fabs(A[i * N + k]); r = i; }
      perm[k] = r;
      if (!(best > tiny_pivot<T>())) atomicOr(status, kDevSingular);
      if (r != k) {
#pragma unroll 1
        for (int j = 0; j < N; ++j) {
          const T t = A[k * N + j];
          A[k * N + j] = A[r * N + j];
          A[r * N + j] = t;
        }
      }
      const T inv = (T)1 / A[k * N + k];
#pragma unroll 1
      for (int j = 0; j < N; ++j)
        if (j != k) A[k * N + j] *= inv;
      A[k * N + k] = inv;
#pragma unroll 1
      for (int i = 0; i < N; ++i) {
        if (i == k) continue;
        const T fct = A[i * N + k];
#pragma unroll 1
        for (int j = 0; j < N; ++j)
          if (j != k) A[i * N + j] -= fct * A[k * N + j];
        A[i * N + k] = -fct * inv;
      }
    }
#pragma unroll 1
    for (int k = N - 1; k >= 0; --k) {
      const int r = perm[k];
      if (r == k) continue;
#pragma unroll 1
      for (int i = 0; i < N; ++i) {
        const T t = A[i * N + k];
        A[i * N + k] = A[i * N + r];
        A[i * N + r] = t;
      }
    }
  }
  char* out = L::s_at(rec, m);
  char* outx = L::x_at((char*)rec + nmem * (long long)L::kStaged, m);
  T* ai = L::ainv(outx);
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int i = 0; i < N; ++i) ai[j * N + i] = A[i * N + j];
  if (Y && rhs.bvol) {   // y = A^{-1} b (the sweep's apply, done here)
    T b[N];
#pragma unroll
    for (int j = 0; j < N; ++j) b[j] = rhs_b<P, T>(rhs, ft, nds, nx, ny, E, d, e, j, bits, mu, eta);
    T* yo = rhs.y + (size_t)m * L::kYStride;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T yi = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) yi += A[i * N + j] * b[j];
      yo[i] = yi;
    }
  }
  unsigned faces = 0xffffffffu;
  int slot = 0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (!(bits & (1u << f)) || nb_elem(nx, ny, e, f) < 0) continue;
    T* W = L::slot(out, outx, slot);
    faces = (faces & ~(0xffu << (8 * slot))) | ((unsigned)f << (8 * slot));
    ++slot;
#pragma unroll
    for (int t = 0; t < Q; ++t)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        T w = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) w += A[i * N + face_dof<P>(f, a)] * Cin[f][a][t];
        W[t * N + i] = w;
      }
  }
  *reinterpret_cast<uint4*>(out) = make_uint4((unsigned)e, (unsigned)bits, faces, 0u);
  return bad;
}

template <int P, typename T, bool Y>
__global__ void __launch_bounds__(128)
factor_kernel(long long nmem, const uint32_t* __restrict__ code, const uint16_t* __restrict__ finfo,
              const double* __restrict__ omega, const double* __restrict__ sigma_t,
              const T* __restrict__ Mm, const T* __restrict__ Gxm, const T* __restrict__ Gym,
              const T* __restrict__ nds, FaceTab<T> ft, FaceLL<T> fll, int nx, int ny, long long E,
              T* __restrict__ rec, unsigned int* status, unsigned int* piv_count, unsigned int* piv_list,
              int force_pivot, RhsArgs<T> rhs) {
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= nmem) return;
  const bool bad = factor_task<P, T, false, Y>(m, nmem, code, finfo, omega, sigma_t, Mm, Gxm, Gym, nds, ft,
                                               fll, nx, ny, E, rec, status, rhs);
  if (bad || force_pivot) pivot_list_append(piv_count, piv_list, m);
}

// Fallback for the tasks the guard listed: the same assembly, Gauss-Jordan with partial
// pivoting, the record rewritten.  Grid-stride over the list (its length is read on the
// device, so the launch needs no host synchronisation); whole matrices per thread live in
// local memory, which is acceptable for the few tasks that come here.
template <int P, typename T>
__global__ void __launch_bounds__(128)
factor_pivot_kernel(long long nmem, const uint32_t* __restrict__ code, const uint16_t* __restrict__ finfo,
                    const double* __restrict__ omega, const double* __restrict__ sigma_t,
                    const T* __restrict__ Mm, const T* __restrict__ Gxm, const T* __restrict__ Gym,
                    const T* __restrict__ nds, FaceTab<T> ft, FaceLL<T> fll, int nx, int ny, long long E,
                    T* __restrict__ rec, unsigned int* status, const unsigned int* piv_count,
                    const unsigned int* __restrict__ piv_list, RhsArgs<T> rhs) {
  const long long cnt = (long long)*piv_count;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cnt && t < nmem;
       t += (long long)gridDim.x * blockDim.x)
    if (VEF_IN_RANGE(piv_list[t], nmem, status))
      factor_task<P, T, true, true>((long long)piv_list[t], nmem, code, finfo, omega, sigma_t, Mm, Gxm, Gym, nds,
                                    ft, fll, nx, ny, E, rec, status, rhs);
}

// Element-major factorisation (used for p >= 3, where a whole element matrix per thread
// spills).  One CTA per element stages M, Gx, Gy and the face normals in shared memory
// once and walks the element's directions, so the direction-independent element data is
// read from memory once instead of D times.  A task (one direction) is held by LPU lanes,
// each owning RPL rows of A (row i on lane i mod LPU, slot i / LPU).  Gauss-Jordan step k
// broadcasts the unscaled pivot row r = A[k][:] from its owner lane, and every row
// applies one FMA per entry, row[j] += beta r[j], with beta = -A[i][k] / r[k] on the other
// rows and beta = 1/r[k] - 1 on the pivot row itself (which turns it into r / r[k]);
// column k then becomes -A[i][k] / r[k], or 1 / r[k] on the pivot row.  With several rows
// per lane the reciprocal and the broadcast are shared by RPL rows' FMAs.
template <int P, typename T> struct ElemShape;
// EPC elements per CTA: at p = 3 in FP64 a warp holds 8 tasks, and the level-symmetric sets
// have D = 4 (mod 8) directions for S4 and S12, so one element per CTA would leave half a
// warp of padding tasks computing; two elements per CTA fill every warp (2 D = 0 mod 8).
// FP64 is bound by its FP64 pipe, so four rows per lane share each pivot-row broadcast.
// FP32 is bound by latency instead (four register-limited warps per scheduler at four rows
// per lane): two rows per lane halve the registers, so six CTAs fit per SM.
template <> struct ElemShape<3, double> { static constexpr int RPL = 4, LPU = 4, EPC = 2, MINB = 1; };
template <> struct ElemShape<3, float> { static constexpr int RPL = 2, LPU = 8, EPC = 4, MINB = 6; };
template <typename T> struct ElemShape<4, T> { static constexpr int RPL = 2, LPU = 13, EPC = 1, MINB = 1; };

template <int P, typename T, bool Y>
__global__ void __launch_bounds__(128, ElemShape<P, T>::MINB)
factor_elem_kernel(int D, long long E, const int* __restrict__ member_of, const uint16_t* __restrict__ finfo,
                   const double* __restrict__ omega, const double* __restrict__ sigma_t,
                   const T* __restrict__ Mm, const T* __restrict__ Gxm, const T* __restrict__ Gym,
                   const T* __restrict__ nds, FaceTab<T> ft, int nx, int ny, long long nmem,
                   T* __restrict__ rec, unsigned int* status, unsigned int* piv_count,
                   unsigned int* piv_list, int force_pivot, RhsArgs<T> rhs) {
  constexpr int Q = P + 1, N = Q * Q, NQ = P + 2;
  constexpr int RPL = ElemShape<P, T>::RPL, LPU = ElemShape<P, T>::LPU, UPW = 32 / LPU, EPC = ElemShape<P, T>::EPC;
  constexpr int LD = N + 1;                  // padded shared-memory row stride
  constexpr int CPL = (Q * Q + LPU - 1) / LPU;   // inflow-coupling entries computed per lane
  constexpr unsigned FULL = 0xffffffffu;
  using L = Rec<P, T>;
  __shared__ T sM[EPC][N * LD], sX[EPC][N * LD], sY[EPC][N * LD];   // sigma_t M (scaled once), Gx, Gy
  __shared__ T sN[EPC][4 * NQ * 2];
  __shared__ T sLL[Q][Q][NQ];          // l_a(s_k) l_t(s_k): face basis products
  __shared__ T sW[NQ];                 // face Gauss weights
  __shared__ T sC[4][UPW][4][NQ];      // per warp and task: w_k Omega . (n ds)_k of each face
  const long long e0 = (long long)blockIdx.x * EPC;
  const int ne = (int)min((long long)EPC, E - e0);   // elements of this CTA
  const int tid = threadIdx.x;
  for (int idx = tid; idx < ne * N * N; idx += blockDim.x) {
    const int el = idx / (N * N), r = (idx / N) % N, j = idx % N;
    const size_t g = (size_t)e0 * N * N + idx;
    sM[el][r * LD + j] = (T)sigma_t[e0 + el] * Mm[g];
    sX[el][r * LD + j] = Gxm[g];
    sY[el][r * LD + j] = Gym[g];
  }
  for (int idx = tid; idx < ne * 4 * NQ * 2; idx += blockDim.x)
    sN[idx / (4 * NQ * 2)][idx % (4 * NQ * 2)] = nds[(size_t)e0 * 4 * NQ * 2 + idx];
  for (int idx = tid; idx < Q * Q * NQ; idx += blockDim.x) {
    const int qa = idx / (Q * NQ), qt = (idx / NQ) % Q, kk = idx % NQ;
    sLL[qa][qt][kk] = ft.l[qa][kk] * ft.l[qt][kk];
  }
  if (tid < NQ) sW[tid] = ft.w[tid];
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int u = lane / LPU, li = lane % LPU, base = u * LPU;
  const int uc = u < UPW ? u : UPW - 1;   // lanes past the last task read a valid slot
  char* recx = (char*)rec + nmem * (long long)L::kStaged;
  // tasks t = el D + d of the CTA's elements, UPW per warp and round
  const int ntask = ne * D;
  for (int t0 = warp * UPW; t0 < ntask; t0 += nwarps * UPW) {
    const int t = t0 + u;
    bool valid = u < UPW && t < ntask;
    const int tt = valid ? t : 0, el = tt / D, dd = tt % D;
    const long long e = e0 + el;
    const T mu = (T)omega[2 * dd], eta = (T)omega[2 * dd + 1];
    const uint16_t bits = finfo[(size_t)dd * E + e];
    // face coefficients of this task, once: its LPU lanes share the 4 NQ entries
    __syncwarp();
    for (int q = li; u < UPW && q < 4 * NQ; q += LPU) {
      const int f = q / NQ, kk = q % NQ;
      sC[warp][u][f][kk] = sW[kk] * (mu * sN[el][(f * NQ + kk) * 2] + eta * sN[el][(f * NQ + kk) * 2 + 1]);
    }
    __syncwarp();
    // assemble the owned rows: sigma_t M - mu Gx - eta Gy ...
    T row[RPL][N];
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      const int i = li + LPU * r;
#pragma unroll
      for (int j = 0; j < N; ++j)
        row[r][j] = i < N ? fma(-eta, sY[el][i * LD + j], fma(-mu, sX[el][i * LD + j], sM[el][i * LD + j])) : (T)0;
    }
    // ... plus the outflow face terms: row a of face f's matrix sum_k max(c_k, 0) l_a l_t is
    // formed on lane a of the task and shuffled to the lane that owns face node a (faces
    // without an outflow point in any of the warp's tasks are skipped)
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      bool out_f = false;
#pragma unroll
      for (int k = 0; k < NQ; ++k) out_f = out_f || sC[warp][uc][f][k] > (T)0;
      if (!__any_sync(FULL, valid && out_f)) continue;
      const int fa = li < Q ? li : Q - 1;   // lanes past the face's p+1 rows form a copy
      T fo[Q];
#pragma unroll
      for (int t = 0; t < Q; ++t) fo[t] = 0;
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        const T s = sC[warp][uc][f][k];
        const T sp = s > (T)0 ? s : (T)0;
#pragma unroll
        for (int t = 0; t < Q; ++t) fo[t] = fma(sp, sLL[fa][t][k], fo[t]);
      }
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = li + LPU * r;
        const int ia = i % Q, ib = i / Q;
        int pos = -1;
        if (i < N) {
          if (f == 0 && ib == 0) pos = ia;
          if (f == 1 && ia == P) pos = ib;
          if (f == 2 && ib == P) pos = ia;
          if (f == 3 && ia == 0) pos = ib;
        }
        if (!__any_sync(FULL, pos >= 0)) continue;
        const int src = (base + (pos > 0 ? pos : 0)) & 31;
#pragma unroll
        for (int t = 0; t < Q; ++t) {
          const T v = __shfl_sync(FULL, fo[t], src);
          if (pos >= 0) row[r][face_dof<P>(f, t)] += v;
        }
      }
    }
    // row scales of the owned rows for the pivot guard (integer operations only)
    int scl[RPL];
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      int mx = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) mx = max(mx, PivotFloor<T>::mag(row[r][j]));
      scl[r] = mx;
    }
    bool bad = false;
    // in-place Gauss-Jordan over the task's LPU lanes (no pivoting; the owner of row k
    // checks its pivot against the row's scale)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int owner = k % LPU, slot = k / LPU;
      T pr[N];
#pragma unroll
      for (int j = 0; j < N; ++j) pr[j] = __shfl_sync(FULL, row[slot][j], (base + owner) & 31);
      if (li == owner) bad = bad || small_pivot<T>(pr[k], scl[slot]);
      const T inv = pivot_rcp(pr[k]);
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = li + LPU * r;
        const T aik = row[r][k];
        const T beta = (i == k) ? inv - (T)1 : -aik * inv;
#pragma unroll
        for (int j = 0; j < N; ++j)
          if (j != k) row[r][j] = fma(beta, pr[j], row[r][j]);
        row[r][k] = (i == k) ? inv : -aik * inv;
      }
    }
    // records: A^{-1} column-major, then the W slots of the interior inflow faces
    const long long m = valid ? (long long)member_of[(size_t)dd * E + e] : 0;
    valid = valid && VEF_IN_RANGE(m, nmem, status);
    char* out = L::s_at(rec, m);
    char* outx = L::x_at(recx, m);
    if (valid) {
      T* ai = L::ainv(outx);
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = li + LPU * r;
        if (i >= N) continue;
#pragma unroll
        for (int j = 0; j < N; ++j) ai[j * N + i] = row[r][j];
      }
    }
    if constexpr (Y) {   // y = A^{-1} b for the owned rows (the sweep's apply, done here)
      T bown[RPL], yr[RPL];
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = li + LPU * r;
        bown[r] = (valid && i < N) ? rhs_b<P, T>(rhs, ft, nds, nx, ny, E, dd, (int)e, i, bits, mu, eta) : (T)0;
        yr[r] = 0;
      }
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const T bj = __shfl_sync(FULL, bown[j / LPU], (base + j % LPU) & 31);
#pragma unroll
        for (int r = 0; r < RPL; ++r) yr[r] = fma(row[r][j], bj, yr[r]);
      }
      if (valid) {
        T* yo = rhs.y + (size_t)m * L::kYStride;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          const int i = li + LPU * r;
          if (i < N) yo[i] = yr[r];
        }
      }
    }
    unsigned faces = 0xffffffffu;
    int nslot = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const bool use = valid && (bits & (1u << f)) && nb_elem(nx, ny, (int)e, f) >= 0;
      if (!__any_sync(FULL, use)) continue;
      // Cin_f[a][t] = sum_k min(c_k, 0) l_a(s_k) l_t(s_k), entries q = a Q + t spread over
      // the task's lanes, then gathered
      T cmine[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int q = li + LPU * c;
        T v = 0;
        if (q < Q * Q) {
          const int qa = q / Q, qt = q % Q;
#pragma unroll
          for (int k = 0; k < NQ; ++k) {
            const T s = sC[warp][uc][f][k];
            v = fma(s < (T)0 ? s : (T)0, sLL[qa][qt][k], v);
          }
        }
        cmine[c] = v;
      }
      T W[RPL][Q];
#pragma unroll
      for (int r = 0; r < RPL; ++r)
#pragma unroll
        for (int t = 0; t < Q; ++t) W[r][t] = 0;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
#pragma unroll
        for (int t = 0; t < Q; ++t) {
          const int q = a * Q + t;
          const T cat = __shfl_sync(FULL, cmine[q / LPU], (base + q % LPU) & 31);
#pragma unroll
          for (int r = 0; r < RPL; ++r) W[r][t] = fma(row[r][face_dof<P>(f, a)], cat, W[r][t]);
        }
      }
      if (use) {
        T* Wo = L::slot(out, outx, nslot);
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          const int i = li + LPU * r;
          if (i >= N) continue;
#pragma unroll
          for (int t = 0; t < Q; ++t) Wo[t * N + i] = W[r][t];
        }
        faces = (faces & ~(0xffu << (8 * nslot))) | ((unsigned)f << (8 * nslot));
        ++nslot;
      }
    }
    if (valid && li == 0) *reinterpret_cast<uint4*>(out) = make_uint4((unsigned)e, (unsigned)bits, faces, 0u);
    // a task any of whose lanes saw a small pivot goes to the pivoted fallback
    const unsigned bal = __ballot_sync(FULL, bad || force_pivot);
    if (valid && li == 0 && ((bal >> base) & ((1u << LPU) - 1u))) pivot_list_append(piv_count, piv_list, m);
  }
}

// FP64 element matrix and inflow couplings of every (element, direction), for the FP64
// residual of the mixed-precision defect correction: per task [A (n x n, column-major)]
// [Cin of W slots 0..3 ((p+1) x (p+1), row a = own face node, column t = neighbour's)].
// Element-major like factor_elem_kernel: one CTA per element holds M, Gx, Gy, the
// normals and the face products l_a(s_k) l_t(s_k) in shared memory.  A task takes
// LPU = max(n, 4(p+1)) lanes: lane i < n assembles row i of the volume part, lane
// f (p+1) + a < 4 (p+1) forms row a of face f's outflow and inflow matrices, and the
// outflow rows are shuffled to the lanes owning those matrix rows.  Every lane does
// useful FP64 work and every store of A is coalesced.
template <int P>
__global__ void __launch_bounds__(128)
assemble64_kernel(int D, long long E, const int* __restrict__ member_of, const uint16_t* __restrict__ finfo,
                  const double* __restrict__ omega, const double* __restrict__ sigma_t,
                  const double* __restrict__ Mm, const double* __restrict__ Gxm,
                  const double* __restrict__ Gym, const double* __restrict__ nds, FaceTab<double> ft,
                  int nx, int ny, double* __restrict__ out) {
  constexpr int Q = P + 1, N = Q * Q, NQ = P + 2, B = N * N + 4 * Q * Q;
  constexpr int LPU = N > 4 * Q ? N : 4 * Q;
  constexpr int UPW = 32 / LPU;
  constexpr int LD = N + 1;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ double sM[N * LD], sX[N * LD], sY[N * LD];
  __shared__ double sN[4 * NQ * 2];
  __shared__ double sLL[Q][Q][NQ];
  const long long e = blockIdx.x;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < N * N; idx += blockDim.x) {
    const int r = idx / N, j = idx % N;
    const size_t g = (size_t)e * N * N + idx;
    sM[r * LD + j] = Mm[g];
    sX[r * LD + j] = Gxm[g];
    sY[r * LD + j] = Gym[g];
  }
  for (int idx = tid; idx < 4 * NQ * 2; idx += blockDim.x) sN[idx] = nds[(size_t)e * 4 * NQ * 2 + idx];
  for (int idx = tid; idx < Q * Q * NQ; idx += blockDim.x) {
    const int qa = idx / (Q * NQ), qt = (idx / NQ) % Q, k = idx % NQ;
    sLL[qa][qt][k] = ft.l[qa][k] * ft.l[qt][k];
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int u = lane / LPU, li = lane % LPU, base = u * LPU;
  const double st = sigma_t[e];
  const int ia = li % Q, ib = li / Q;                 // node of row li (li < n)
  const int ff = li / Q, fa = li % Q;                 // face row of lane li (li < 4 (p+1))
  for (int d0 = warp * UPW; d0 < D; d0 += nwarps * UPW) {
    const int d = d0 + u;
    const bool valid = u < UPW && d < D;
    const int dd = valid ? d : 0;
    const double mu = omega[2 * dd], eta = omega[2 * dd + 1];
    const uint16_t bits = finfo[(size_t)dd * E + e];
    double row[N];
#pragma unroll
    for (int j = 0; j < N; ++j)
      row[j] = li < N ? st * sM[li * LD + j] - mu * sX[li * LD + j] - eta * sY[li * LD + j] : 0.0;
    double fo[Q], ci[Q];
#pragma unroll
    for (int t = 0; t < Q; ++t) fo[t] = ci[t] = 0.0;
    if (li < 4 * Q) {
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        const double c = ft.w[k] * (mu * sN[(ff * NQ + k) * 2] + eta * sN[(ff * NQ + k) * 2 + 1]);
        const double cp = c > 0.0 ? c : 0.0, cm = c < 0.0 ? c : 0.0;
#pragma unroll
        for (int t = 0; t < Q; ++t) {
          fo[t] = fma(cp, sLL[fa][t][k], fo[t]);
          ci[t] = fma(cm, sLL[fa][t][k], ci[t]);
        }
      }
    }
    // outflow face rows onto the matrix rows they belong to
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      int pos = -1;
      if (f == 0 && ib == 0) pos = ia;
      if (f == 1 && ia == P) pos = ib;
      if (f == 2 && ib == P) pos = ia;
      if (f == 3 && ia == 0) pos = ib;
      const int src = (base + f * Q + (pos > 0 ? pos : 0)) & 31;
#pragma unroll
      for (int t = 0; t < Q; ++t) {
        const double v = __shfl_sync(FULL, fo[t], src);
        if (li < N && pos >= 0) row[face_dof<P>(f, t)] += v;
      }
    }
    if (!valid) continue;
    double* blk = out + (long long)member_of[(size_t)d * E + e] * B;
    if (li < N) {
#pragma unroll
      for (int j = 0; j < N; ++j) blk[j * N + li] = row[j];
    }
    if (li < 4 * Q && (bits & (1u << ff)) && nb_elem(nx, ny, (int)e, ff) >= 0) {
      int slot = 0;
      for (int g = 0; g < ff; ++g)
        if ((bits & (1u << g)) && nb_elem(nx, ny, (int)e, g) >= 0) ++slot;
      double* C = blk + N * N + slot * Q * Q + fa * Q;
#pragma unroll
      for (int t = 0; t < Q; ++t) C[t] = ci[t];
    }
  }
}

// Thread-per-task form of the FP64 assembly for p <= 2, where a whole element system
// fits in one thread's registers and every FP64 instruction is useful on all lanes (the
// element-major form wastes lanes on the face rows at these sizes).  Same output layout.
template <int P>
__global__ void __launch_bounds__(128)
assemble64_thread_kernel(long long nmem, const uint32_t* __restrict__ code, const uint16_t* __restrict__ finfo,
                         const double* __restrict__ omega, const double* __restrict__ sigma_t,
                         const double* __restrict__ Mm, const double* __restrict__ Gxm,
                         const double* __restrict__ Gym, const double* __restrict__ nds, FaceTab<double> ft,
                         int nx, int ny, long long E, double* __restrict__ out) {
  constexpr int Q = P + 1, N = Q * Q, NQ = P + 2, B = N * N + 4 * Q * Q;
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= nmem) return;
  const uint32_t c = code[m];
  const int d = (int)(c >> 22), e = (int)(c & 0x3fffffu);
  const double mu = omega[2 * d], eta = omega[2 * d + 1], st = sigma_t[e];
  const uint16_t bits = finfo[(size_t)d * E + e];
  double* blk = out + m * (long long)B;
  const double* Me = Mm + (size_t)e * N * N;
  const double* Xe = Gxm + (size_t)e * N * N;
  const double* Ye = Gym + (size_t)e * N * N;
  double A[N * N];   // column-major
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) A[j * N + i] = st * Me[i * N + j] - mu * Xe[i * N + j] - eta * Ye[i * N + j];
  int slot = 0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    double cp[NQ], cm[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const double* v = nds + (((size_t)e * 4 + f) * NQ + k) * 2;
      const double sv = ft.w[k] * (mu * v[0] + eta * v[1]);
      cp[k] = sv > 0.0 ? sv : 0.0;
      cm[k] = sv < 0.0 ? sv : 0.0;
    }
    const bool inflow_nb = (bits & (1u << f)) && nb_elem(nx, ny, e, f) >= 0;
    double* C = blk + N * N + slot * Q * Q;
#pragma unroll
    for (int a = 0; a < Q; ++a)
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        double vo = 0, vi = 0;
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
          const double ll = ft.l[a][k] * ft.l[b][k];
          vo += cp[k] * ll;
          vi += cm[k] * ll;
        }
        A[face_dof<P>(f, b) * N + face_dof<P>(f, a)] += vo;
        if (inflow_nb) C[a * Q + b] = vi;
      }
    if (inflow_nb) ++slot;
  }
#pragma unroll
  for (int q = 0; q < N * N; ++q) blk[q] = A[q];
}

// Trace system of a coupled element group.  Member a of a group solves
//     psi_a = z_a - sum_{(a,f)} W_{a,f} tau_{a,f},
// where z_a = A_a^{-1} b_a minus the couplings to elements outside the group, and the
// sum runs over the faces f of a that are inflow somewhere and shared with another
// member b; tau_{a,f} holds b's values at the p+1 nodes of its face opposite f.  Taking
// those traces of the member equations gives the closed system
//     (I + R) tau = P z,   R[(a,f,s), (b,g,t)] = W_{b,g}[face_dof(opp f, s)][t],
// which is the element block system of the group (the upwind weak form with the group's
// internal upwind traces as unknowns) reduced to its interface.  One CTA per group forms
// I + R in shared memory and inverts it in place (Gauss-Jordan with partial pivoting, in
// FP64); the inverse is stored column-major.  Trace unknowns are numbered by member, then
// face, then face node; the sweep numbers them the same way.
template <int P, typename T>
__global__ void __launch_bounds__(128)
group_factor_kernel(int g0, const int* __restrict__ grp_slot, const int* __restrict__ grp_nt,
                    const long long* __restrict__ grp_toff, const int* __restrict__ slot_first,
                    const int* __restrict__ slot_count, const uint32_t* __restrict__ member_nbpos,
                    const T* __restrict__ rec, long long nmem, T* __restrict__ grec,
                    unsigned int* status) {
  constexpr int Q = P + 1, N = Q * Q;
  constexpr int GM = group_direct_members(P);
  constexpr int NC = kGroupMaxTrace / Q + 1;
  using L = Rec<P, T>;
  extern __shared__ __align__(16) double gsm[];
  __shared__ uint32_t cpl[NC];
  __shared__ int perm[kGroupMaxTrace];
  __shared__ double colk[kGroupMaxTrace];
  __shared__ int piv_row, ncpl;
  const int g = g0 + (int)blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const int sl = grp_slot[g], nt = grp_nt[g];
  const int first = slot_first[sl], m = slot_count[sl];
  const char* recx = (const char*)rec + nmem * (long long)L::kStaged;
  double* Mx = gsm;   // nt x nt, row-major
  if (tid == 0) {
    int c = 0;
    for (int a = 0; a < m && a < GM; ++a) {
      const uint4 info = *reinterpret_cast<const uint4*>(L::s_at(rec, first + a));
      const uint32_t nbp = member_nbpos[first + a];
      for (int f = 0; f < 4; ++f) {
        if (!((info.y >> f) & 1u) || !((info.y >> (4 + f)) & 1u)) continue;
        const int s = rec_slot_of(info.z, f);
        if (c < NC && s >= 0) cpl[c] = (uint32_t)a | ((uint32_t)f << 8) | (((nbp >> (8 * f)) & 0xffu) << 16) |
                                       ((uint32_t)s << 24);
        ++c;
      }
    }
    ncpl = c;
  }
  __syncthreads();
  if (ncpl * Q != nt) {   // schedule and records disagree: leave the group to the iteration
    if (tid == 0) atomicOr(status, kDevSingular);
    return;
  }
  // rows by warp, columns by lane (no integer division by the runtime size)
  const int lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  for (int r = wid; r < nt; r += nw) {
    const uint32_t c1 = cpl[r / Q];
    const int b = (int)((c1 >> 16) & 0xffu), f = (int)((c1 >> 8) & 0xffu);
    for (int col = lane; col < nt; col += 32) {
      const uint32_t c2 = cpl[col / Q];
      double v = r == col ? 1.0 : 0.0;
      if ((int)(c2 & 0xffu) == b) {
        const T* W = L::slot(L::s_at(rec, first + b), L::x_at(recx, first + b), (int)(c2 >> 24));
        v += (double)W[(col % Q) * N + face_dof<P>((f + 2) & 3, r % Q)];
      }
      Mx[r * nt + col] = v;
    }
  }
  for (int k = 0; k < nt; ++k) {
    __syncthreads();
    if (tid < 32) {   // pivot: largest |entry| of column k on or below the diagonal
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < nt; i += 32) {
        const double v = fabs(Mx[i * nt + k]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        piv_row = bi;
        perm[k] = bi;
        if (!(best > 1e-300)) atomicOr(status, kDevSingular);
      }
    }
    __syncthreads();
    const int pr = piv_row;
    if (pr != k)
      for (int j = tid; j < nt; j += nth) {
        const double t = Mx[k * nt + j];
        Mx[k * nt + j] = Mx[pr * nt + j];
        Mx[pr * nt + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / Mx[k * nt + k];
    for (int i = tid; i < nt; i += nth) colk[i] = Mx[i * nt + k];
    __syncthreads();
    for (int j = tid; j < nt; j += nth) Mx[k * nt + j] = j == k ? inv : Mx[k * nt + j] * inv;
    __syncthreads();
    for (int i = wid; i < nt; i += nw) {
      if (i == k) continue;
      const double ci = colk[i];
      for (int j = lane; j < nt; j += 32)
        Mx[i * nt + j] = j == k ? -ci * inv : fma(-ci, Mx[k * nt + j], Mx[i * nt + j]);
    }
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = nt - 1; k >= 0; --k) {
    __syncthreads();
    const int pr = perm[k];
    if (pr != k)
      for (int i = tid; i < nt; i += nth) {
        const double t = Mx[i * nt + k];
        Mx[i * nt + k] = Mx[i * nt + pr];
        Mx[i * nt + pr] = t;
      }
  }
  __syncthreads();
  T* out = grec + grp_toff[g];
  for (int j = wid; j < nt; j += nw)
    for (int r = lane; r < nt; r += 32) out[j * nt + r] = (T)Mx[r * nt + j];
}

// Small trace systems (nt <= NTB <= 32): one warp per group, lane r holds row r of
// I + R in registers; the pivot search is a warp argmax, row interchanges and the
// pivot-row broadcast are shuffles.  Same algorithm as group_factor_kernel.
template <int P, typename T, int NTB>
__global__ void __launch_bounds__(128)
group_factor_warp_kernel(int g0, int g1, const int* __restrict__ grp_slot, const int* __restrict__ grp_nt,
                         const long long* __restrict__ grp_toff, const int* __restrict__ slot_first,
                         const int* __restrict__ slot_count, const uint32_t* __restrict__ member_nbpos,
                         const T* __restrict__ rec, long long nmem, T* __restrict__ grec,
                         unsigned int* status) {
  constexpr int Q = P + 1, N = Q * Q;
  constexpr int NCW = NTB / Q + 1;
  constexpr unsigned FULL = 0xffffffffu;
  using L = Rec<P, T>;
  __shared__ uint32_t cpl_s[4][NCW];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int g = g0 + (int)blockIdx.x * (int)(blockDim.x >> 5) + wib;
  if (g >= g1) return;   // the whole warp
  const int sl = grp_slot[g], nt = grp_nt[g];
  const int first = slot_first[sl], m = slot_count[sl];   // m <= 32 for a direct group
  const char* recx = (const char*)rec + nmem * (long long)L::kStaged;
  uint32_t* cpl = cpl_s[wib];
  uint4 info = make_uint4(0u, 0u, 0xffffffffu, 0u);
  uint32_t nbp = 0xffffffffu;
  if (lane < m) {
    info = *reinterpret_cast<const uint4*>(L::s_at(rec, first + lane));
    nbp = member_nbpos[first + lane];
  }
  const unsigned mine = lane < m ? (unsigned)__popc(info.y & (info.y >> 4) & 0xfu) : 0u;
  unsigned incl = mine;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned v = __shfl_up_sync(FULL, incl, off);
    if (lane >= off) incl += v;
  }
  const int total = (int)__shfl_sync(FULL, incl, 31);
  if (total * Q != nt || nt > NTB) {   // schedule and records disagree
    if (lane == 0) atomicOr(status, kDevSingular);
    return;
  }
  if (lane < m) {
    unsigned c = incl - mine;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      if (!((info.y >> f) & 1u) || !((info.y >> (4 + f)) & 1u)) continue;
      cpl[c++] = (uint32_t)lane | ((uint32_t)f << 8) | (((nbp >> (8 * f)) & 0xffu) << 16) |
                 ((uint32_t)rec_slot_of(info.z, f) << 24);
    }
  }
  __syncwarp();
  double row[NTB];
  {
    const uint32_t c1 = cpl[(lane < nt ? lane : 0) / Q];
    const int b = (int)((c1 >> 16) & 0xffu), f = (int)((c1 >> 8) & 0xffu), s = lane % Q;
#pragma unroll
    for (int j = 0; j < NTB; ++j) {
      double v = (lane == j && lane < nt) ? 1.0 : 0.0;
      if (lane < nt && j < nt) {
        const uint32_t c2 = cpl[j / Q];
        if ((int)(c2 & 0xffu) == b) {
          const T* W = L::slot(L::s_at(rec, first + b), L::x_at(recx, first + b), (int)(c2 >> 24));
          v += (double)W[(j % Q) * N + face_dof<P>((f + 2) & 3, s)];
        }
      }
      row[j] = v;
    }
  }
  int myperm = lane;
#pragma unroll
  for (int k = 0; k < NTB; ++k) {
    if (k >= nt) break;
    double best = (lane >= k && lane < nt) ? fabs(row[k]) : -1.0;
    int bi = lane;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ob = __shfl_xor_sync(FULL, best, off);
      const int oi = __shfl_xor_sync(FULL, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0 && !(best > 1e-300)) atomicOr(status, kDevSingular);
    if (lane == k) myperm = bi;
    if (bi != k) {
      const int src = lane == k ? bi : (lane == bi ? k : lane);
#pragma unroll
      for (int j = 0; j < NTB; ++j) row[j] = __shfl_sync(FULL, row[j], src);
    }
    double pr[NTB];
#pragma unroll
    for (int j = 0; j < NTB; ++j) pr[j] = __shfl_sync(FULL, row[j], k);
    const double inv = 1.0 / pr[k];
    const double aik = row[k];
    const double beta = lane == k ? inv - 1.0 : -aik * inv;
#pragma unroll
    for (int j = 0; j < NTB; ++j)
      if (j != k) row[j] = fma(beta, pr[j], row[j]);
    row[k] = lane == k ? inv : -aik * inv;
  }
  // undo the row interchanges as column interchanges, last first
#pragma unroll
  for (int k = NTB - 1; k >= 0; --k) {
    if (k >= nt) continue;
    const int pk = __shfl_sync(FULL, myperm, k);
    if (pk == k) continue;
    const double vk = row[k];
    double vp = 0.0;
#pragma unroll
    for (int j = 0; j < NTB; ++j)
      if (j == pk) vp = row[j];
#pragma unroll
    for (int j = 0; j < NTB; ++j)
      if (j == pk) row[j] = vk;
    row[k] = vp;
  }
  if (lane < nt) {
    T* out = grec + grp_toff[g];
#pragma unroll
    for (int j = 0; j < NTB; ++j)
      if (j < nt) out[j * nt + lane] = (T)row[j];
  }
}

template <int P, typename T>
static vef_status launch_group_factor(Schedule& S, const void* rec, cudaStream_t stream, unsigned int* status) {
  if (S.ngroups == 0) return VEF_OK;
  void** gp = std::is_same<T, double>::value ? &S.grec64 : &S.grec32;
  if (!*gp) {
    size_t cap = 0;
    vef_status st = ensure_buffer(gp, &cap, (size_t)std::max(1LL, S.grec_elems) * sizeof(T));
    if (st != VEF_OK) return st;
  }
  // groups are numbered by trace-system size: warps for nt <= 8, 16, 32, one CTA with
  // shared memory sized for the largest for the rest
  const long long* up = S.ngroups_upto;
  const long long lo[3] = {0, up[0], up[1]};
  auto warp_launch = [&](auto kernel, long long a, long long b) -> vef_status {
    if (b <= a) return VEF_OK;
    kernel<<<(unsigned)((b - a + 3) / 4), 128, 0, stream>>>((int)a, (int)b, S.grp_slot, S.grp_nt, S.grp_toff,
                                                           S.slot_first, S.slot_count, S.member_nbpos,
                                                           (const T*)rec, S.members, (T*)*gp, status);
    VEF_CUDA_TRY(cudaGetLastError());
    return VEF_OK;
  };
  vef_status st;
  if ((st = warp_launch(group_factor_warp_kernel<P, T, 8>, lo[0], up[0])) != VEF_OK) return st;
  if ((st = warp_launch(group_factor_warp_kernel<P, T, 16>, lo[1], up[1])) != VEF_OK) return st;
  if ((st = warp_launch(group_factor_warp_kernel<P, T, 32>, lo[2], up[2])) != VEF_OK) return st;
  if (S.ngroups > up[2]) {
    const size_t smem = (size_t)S.max_nt * S.max_nt * sizeof(double);
    VEF_CUDA_TRY(cudaFuncSetAttribute(group_factor_kernel<P, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    group_factor_kernel<P, T><<<(unsigned)(S.ngroups - up[2]), 128, smem, stream>>>(
        (int)up[2], S.grp_slot, S.grp_nt, S.grp_toff, S.slot_first, S.slot_count, S.member_nbpos,
        (const T*)rec, S.members, (T*)*gp, status);
    VEF_CUDA_TRY(cudaGetLastError());
  }
  return VEF_OK;
}

template <int P, typename T>
static vef_status launch_factor(Mesh& M, Schedule& S, const double* sigma_t, bool store_systems,
                                int force_pivot, const FactorRhs* rhs, cudaStream_t stream) {
  void** recp = std::is_same<T, double>::value ? &S.rec64 : &S.rec32;
  if (!*recp) {
    // zero-filled once: the W slots of faces without interior inflow are never written
    // and stay zero (the single-CTA sweep multiplies them by a zero trace)
    size_t cap = 0;
    const size_t bytes = (size_t)S.members * (Rec<P, T>::kStaged + Rec<P, T>::kX);
    vef_status st = ensure_buffer(recp, &cap, bytes);
    if (st != VEF_OK) return st;
    VEF_CUDA_TRY(cudaMemsetAsync(*recp, 0, bytes, stream));
  }
  const T* Mm;
  const T* Gx;
  const T* Gy;
  const T* nds;
  if (std::is_same<T, double>::value) {
    Mm = (const T*)M.Mmat; Gx = (const T*)M.Gx; Gy = (const T*)M.Gy; nds = (const T*)M.nds;
  } else {
    vef_status st = mesh_float_copies(&M, stream);
    if (st != VEF_OK) return st;
    Mm = (const T*)M.Mmat32; Gx = (const T*)M.Gx32; Gy = (const T*)M.Gy32; nds = (const T*)M.nds32;
  }
  if (!std::is_same<T, double>::value && store_systems) {
    constexpr int Q = P + 1, N = Q * Q;
    if (!S.a64) {
      size_t cap = 0;
      vef_status st = ensure_buffer(&S.a64, &cap, (size_t)S.members * (N * N + 4 * Q * Q) * sizeof(double));
      if (st != VEF_OK) return st;
    }
    KTimer kt(&M, VEF_K_FACTOR, stream);
    if constexpr (P >= 3) {
      constexpr int UPW = 32 / (N > 4 * Q ? N : 4 * Q);
      const int warps = std::max(1, std::min(4, (S.D + UPW - 1) / UPW));
      assemble64_kernel<P><<<(unsigned)M.E, 32 * warps, 0, stream>>>(
          S.D, M.E, S.member_of, S.faceinfo, S.omega_dev, sigma_t, M.Mmat, M.Gx, M.Gy, M.nds,
          make_facetab<double>(M.tab), M.nx, M.ny, (double*)S.a64);
    } else {
      assemble64_thread_kernel<P><<<nblk(S.members, 128), 128, 0, stream>>>(
          S.members, S.member_code, S.faceinfo, S.omega_dev, sigma_t, M.Mmat, M.Gx, M.Gy, M.nds,
          make_facetab<double>(M.tab), M.nx, M.ny, M.E, (double*)S.a64);
    }
  }
  if (!S.pivot_list) {
    size_t cap = 0;
    vef_status st = ensure_buffer((void**)&S.pivot_list, &cap, (size_t)S.members * sizeof(unsigned int));
    if (st != VEF_OK) return st;
  }
  RhsArgs<T> ra{};
  if (rhs) {
    vef_status st = ensure_buffer(&M.ybuf, &M.ybuf_cap, (size_t)S.members * Rec<P, T>::kYBytes);
    if (st != VEF_OK) return st;
    ra = RhsArgs<T>{rhs->bvol, rhs->src_aniso, rhs->inflow, M.Mmat, (T*)M.ybuf, M.nbf};
  }
  unsigned int* piv_count = M.dev_status + kStatusPivoted;
  VEF_CUDA_TRY(cudaMemsetAsync(piv_count, 0, sizeof(unsigned int), stream));
  {
  KTimer kt(&M, VEF_K_FACTOR, stream);
  if constexpr (P >= 3) {
    constexpr int UPW = 32 / ElemShape<P, T>::LPU, EPC = ElemShape<P, T>::EPC;
    const int warps = std::max(1, std::min(4, (EPC * S.D + UPW - 1) / UPW));
    auto kern = rhs ? factor_elem_kernel<P, T, true> : factor_elem_kernel<P, T, false>;
    kern<<<(unsigned)((M.E + EPC - 1) / EPC), 32 * warps, 0, stream>>>(
        S.D, M.E, S.member_of, S.faceinfo, S.omega_dev, sigma_t, Mm, Gx, Gy, nds, make_facetab<T>(M.tab),
        M.nx, M.ny, S.members, (T*)*recp, M.dev_status, piv_count, S.pivot_list, force_pivot, ra);
  } else {
    auto kern = rhs ? factor_kernel<P, T, true> : factor_kernel<P, T, false>;
    kern<<<nblk(S.members, 128), 128, 0, stream>>>(
        S.members, S.member_code, S.faceinfo, S.omega_dev, sigma_t, Mm, Gx, Gy, nds,
        make_facetab<T>(M.tab), make_facell<T>(M.tab), M.nx, M.ny, M.E, (T*)*recp, M.dev_status,
        piv_count, S.pivot_list, force_pivot, ra);
  }
  VEF_CUDA_TRY(cudaGetLastError());
  // the listed tasks again, with partial pivoting (the list's length is read on the device)
  int dev = 0, sms = 0;
  VEF_CUDA_TRY(cudaGetDevice(&dev));
  VEF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  factor_pivot_kernel<P, T><<<(unsigned)std::max(1LL, std::min<long long>(nblk(S.members, 128), sms * 2LL)), 128, 0,
                              stream>>>(
      S.members, S.member_code, S.faceinfo, S.omega_dev, sigma_t, Mm, Gx, Gy, nds, make_facetab<T>(M.tab),
      make_facell<T>(M.tab), M.nx, M.ny, M.E, (T*)*recp, M.dev_status, piv_count, S.pivot_list, ra);
  VEF_CUDA_TRY(cudaGetLastError());
  }
  if (S.ngroups == 0) return VEF_OK;
  KTimer kt(&M, VEF_K_GROUP, stream);
  return launch_group_factor<P, T>(S, *recp, stream, M.dev_status);
}


}  // namespace

// instantiation for one DG order (one translation unit per order keeps builds parallel)
vef_status VEF_FACTOR_FN(Mesh* mesh, Schedule* S, const double* sigma_t, int precision,
                         bool store_systems, int force_pivot, const FactorRhs* rhs, cudaStream_t stream) {
  if (precision == VEF_FP64)
    return launch_factor<VEF_FACTOR_P, double>(*mesh, *S, sigma_t, false, force_pivot, rhs, stream);
  return launch_factor<VEF_FACTOR_P, float>(*mesh, *S, sigma_t, store_systems, force_pivot, rhs, stream);
}

}  // namespace vef
