// Shared internal declarations of libvef (host and device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "vef.h"

namespace vef {

constexpr int kMaxP = 4;                 // DG order p in 1..4  -> n <= 25 dofs
constexpr int kMaxM = 4;                 // mesh order m in 1..4
constexpr int kMaxN = (kMaxP + 1) * (kMaxP + 1);
constexpr int kMaxNq = kMaxP + 2;        // quadrature points per direction
constexpr int kMaxD = 1023;              // directions (10 bits in a packed task code)
constexpr long long kMaxE = (1LL << 22); // elements (22 bits in a packed task code)
constexpr double kFourPi = 12.566370614359172953850573533118;

// 1D tables for DG order p: GLL nodes, GL points/weights, Lagrange values and
// derivatives of the GLL basis at the GL points.  Passed to kernels by value.
struct Tab1D {
  int p, np1, nq;
  double gll[kMaxP + 1];
  double gl[kMaxNq];
  double glw[kMaxNq];
  double l[kMaxP + 1][kMaxNq];   // l_a(s_k)
  double dl[kMaxP + 1][kMaxNq];  // l_a'(s_k)
};

// host-side tables (tables.cpp)
void gll_nodes(int m, double* x);                    // m+1 points on [0,1]
void gauss_legendre(int n, double* x, double* w);    // n points, weights sum to 1
void lagrange_eval(int nn, const double* nodes, double x, double* val, double* der);
Tab1D make_tab1d(int p);

// error reporting
void set_last_error(const std::string& msg);
vef_status cuda_fail(cudaError_t err, const char* what);
#define VEF_CUDA_TRY(call)                                        \
  do {                                                            \
    cudaError_t _e = (call);                                      \
    if (_e != cudaSuccess) return ::vef::cuda_fail(_e, #call);    \
  } while (0)

// device status word values written by kernels (bit flags)
enum : unsigned int {
  kDevTimeout = 1u,        // a bounded wait on a staging copy gave up
  kDevNotConverged = 2u,
  kDevNonpositive = 4u,
  kDevSingular = 8u,
  kDevBounds = 16u,        // bounds-checked build: an index outside its array (access skipped)
};
// word of the device status array holding the number of tasks the last factorisation
// refactorised with partial pivoting
constexpr int kStatusPivoted = 6;

// Coupled element groups are solved directly through a trace system precomputed by the
// factorisation (schedule.cpp, factor_impl.cuh) when they have at most this many members
// and trace unknowns; larger groups use the inner block Gauss-Seidel iteration.
__host__ __device__ constexpr int group_direct_members(int p) { return p <= 2 ? 32 : 16; }
constexpr int kGroupMaxTrace = 128;
constexpr int kGroupSmemTrace = 32;   // the trace-system inverse sits in shared memory up to this size

// Shared-memory trace slots one single-CTA sweep of DG order p can hold (sweep.cu).  Slot
// kTraceZero holds zeros and is never written; id kTraceSink marks a face whose values no
// later single-element task reads (nothing is stored); the schedule assigns the others.
int cta_trace_capacity(int p);
constexpr unsigned kTraceZero = 0, kTraceSink = 1, kTraceFirst = 2;

// Per-direction-set schedule: dependency levels, element groups and task chunks.
struct Schedule {
  std::vector<double> omega;   // [D][2] host copy (key)
  std::vector<double> weights; // [D]
  int D = 0;
  int levels = 0;              // max dependency levels over the directions
  long long members = 0;       // == D*E
  int total_levels = 0;        // sum over directions of their level counts
  long long nslots = 0;
  long long coupled_groups = 0;
  long long lagged_points = 0;
  // device arrays
  int* dir_lev0 = nullptr;     // [D+1] first level of each direction in lev_begin
  int* lev_begin = nullptr;    // [total_levels+1] first slot of each level
  int* lev_gbegin = nullptr;   // [total_levels] first coupled-group slot of each level
  int* lev_mbegin = nullptr;   // [total_levels] first member of each level (its singles)
  uint2* member_info = nullptr;  // [members] (element, face bits) in schedule order
  uint32_t* member_nbpos = nullptr;  // [members] per face: in-group position of the neighbour or 255
  int* slot_first = nullptr;   // [nslots] first member index (-1 = padding)
  int* slot_count = nullptr;   // [nslots] members in the group
  // coupled groups solved directly: per slot its group index or -1; per group its slot,
  // the number of trace unknowns nt and the offset of its nt x nt inverse in grec
  int* slot_gid = nullptr;     // [nslots]
  int* grp_slot = nullptr;     // [ngroups]
  int* grp_nt = nullptr;       // [ngroups]
  long long* grp_toff = nullptr;  // [ngroups + 1]
  long long ngroups = 0;
  long long ngroups_upto[3] = {0, 0, 0};  // groups (ordered by nt) with nt <= 8, 16, 32
  long long grec_elems = 0;    // entries of all inverses (grp_toff[ngroups])
  int max_nt = 0;
  void* grec64 = nullptr;      // trace-system inverses (lazily allocated): FP64 and FP32
  void* grec32 = nullptr;
  uint32_t* member_code = nullptr;  // [members] (d << 22) | e, in schedule order
  int* member_of = nullptr;    // [D][E] -> member index
  uint16_t* faceinfo = nullptr;  // [D][E] bits 0-3 inflow face, 4-7 intra-group face, 8-11 outflow to a neighbour
  double* omega_dev = nullptr; // [D][2]
  double* weights_dev = nullptr;  // [D]
  // factor records (lazily allocated): FP64 and FP32 copies
  void* rec64 = nullptr;
  void* rec32 = nullptr;
  void* a64 = nullptr;         // FP64 element matrices + inflow couplings (mixed residual)
  unsigned int* pivot_list = nullptr;  // [members] tasks the pivot guard sent to the fallback
  // which factorisations the records hold (for VEF_REUSE_FACTORS): bit 0 FP64 records,
  // bit 1 FP32 records, bit 2 the stored FP64 element systems
  unsigned factored = 0;
  uint32_t* adj_link = nullptr;  // [members][4] downstream receiver across each face:
                                 // (receiver member << 2) | its W slot, or ~0 (adjoint)
  // Shared-memory trace slots of the single-CTA sweep, per member four 16-bit slot ids:
  // x = the slots to read for the record's W slots 0 and 1 (the donors' face-node values;
  // kTraceZero when the slot is absent or its donor is read from global memory), y / z =
  // the slots the member's own face-node values go to, for faces 0, 1 / 2, 3 (kTraceSink
  // when no later single-element task reads them); w bit 0 when some upwind coupling of
  // the member is read from global memory instead (see cta_trace_capacity), bit 1 when
  // some coupling of the adjoint sweep is (it uses the same slots with the roles of
  // reader and writer swapped).
  uint4* tslot = nullptr;
  int trace_slots = 0;          // slots in use at once (max over directions)
  long long trace_global = 0;   // single-to-single face couplings left to global memory
  ~Schedule();
};

struct KStat {
  long long launches = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
};

struct Mesh {
  int device = 0;
  // per-kernel-class launch counters and optional CUDA-event timing
  bool prof_on = false;
  KStat kstat[VEF_K_COUNT];
  std::vector<cudaEvent_t> event_pool;
  int nx = 0, ny = 0, m = 0, p = 0, n = 0, nq = 0;
  long long E = 0, nbf = 0;
  Tab1D tab{};
  // geometry (device, FP64)
  double* Mmat = nullptr;   // [E][n][n]
  double* Gx = nullptr;     // [E][n][n]
  double* Gy = nullptr;     // [E][n][n]
  double* nds = nullptr;    // [E][4][nq][2] outward n ds (canonical on shared faces)
  float* Mmat32 = nullptr;  // FP32 copies for the mixed path (lazily)
  float* Gx32 = nullptr;
  float* Gy32 = nullptr;
  float* nds32 = nullptr;
  std::vector<double> nds_host;  // host copy for schedule building
  double* ctrl_dev = nullptr;    // [E][(m+1)^2][2] control points
  std::shared_ptr<void> map_tab; // mesh-order Lagrange tables (MapTab, mesh.cu)
  // schedules keyed by direction set
  std::vector<std::unique_ptr<Schedule>> schedules;
  // scratch
  unsigned int* dev_status = nullptr;  // [8]: 0 status bits, 2 max inner iterations, 4 host-set bits
  double* bvol = nullptr;        // [E][n] direction-independent right-hand side
  double* work = nullptr;        // general scratch (phi iterates, reductions)
  size_t work_cap = 0;
  double* work2 = nullptr;
  size_t work2_cap = 0;
  void* ybuf = nullptr;          // [D][E][n] A^{-1} b of the current sweep (FP64 or FP32)
  size_t ybuf_cap = 0;
  int* ready_flags = nullptr;    // [D][bands] band flags of the sweep's fused apply
  size_t ready_cap = 0;
  void* vef_work = nullptr;      // VEF fixed-point iteration: iterates, moments, closures
  size_t vef_work_cap = 0;
  // the HRT multiplier solve's graph of one block of Krylov iterations, with the scratch
  // layout it was captured for
  cudaGraphExec_t hrt_graph = nullptr;
  const void* hrt_graph_work = nullptr;
  long long hrt_graph_nl = -1;
  int hrt_graph_p = 0;
  ~Mesh();
};

// Counts one launch of kernel class k and, when timing is on, brackets it with events
// recorded on the launching stream.
class KTimer {
 public:
  KTimer(Mesh* m, int k, cudaStream_t s);
  ~KTimer();
 private:
  Mesh* m_;
  int k_;
  cudaStream_t s_;
  cudaEvent_t e0_ = nullptr;
};

vef_status ensure_buffer(void** ptr, size_t* cap, size_t bytes);
vef_status mesh_float_copies(Mesh* mesh, cudaStream_t stream);
// Right-hand side of a single transport inversion, applied by the factorisation itself:
// y = A^{-1} b for every task, written in schedule order into the mesh's y buffer, so the
// sweep that follows needs no apply pass.  b = bvol (+ M q_d) minus the boundary inflow.
struct FactorRhs {
  const double* bvol = nullptr;       // [E][n] direction-independent part
  const double* src_aniso = nullptr;  // [D][E][n] anisotropic source or null
  const double* inflow = nullptr;     // [D][nbf][nq] or null (vacuum)
};

// Local factorisation of every (element, direction) system in `precision`.  With
// VEF_MIXED and store_systems, also the FP64 element systems the stored-form residual of
// the defect correction reads (S->a64); without, the residual is formed matrix-free.
// Tasks whose unpivoted elimination meets a small pivot are refactorised with partial
// pivoting (all tasks when force_pivot != 0); their count lands in
// dev_status[kStatusPivoted].
// With rhs non-null, also y = A^{-1} b (see FactorRhs).
vef_status factor_records(Mesh* mesh, Schedule* S, const double* sigma_t, int precision,
                          bool store_systems, int force_pivot, const FactorRhs* rhs,
                          cudaStream_t stream);
Schedule* get_schedule(Mesh* mesh, const double* omega, const double* weights, int D,
                       cudaStream_t stream, vef_status* st);
// Waits for `stream`, reads and clears the handle's device status word, maps it to a status.
vef_status collect_status(Mesh& M, cudaStream_t stream, vef_info* info);

}  // namespace vef

struct vef_mesh_s {
  vef::Mesh impl;
};
