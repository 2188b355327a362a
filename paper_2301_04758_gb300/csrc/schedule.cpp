// Sweep schedule: per-direction upwind dependency graph, its strongly coupled element
// groups and the dependency levels the sweep kernel walks (one cluster per direction).
//
// For direction Omega_d, element e depends on its neighbour across face f when some
// Gauss point of that face is strictly inflow (Omega . n ds < 0); a tangential point
// (Omega . n = 0) counts as outflow.  On straight meshes this graph is the per-quadrant
// diagonal wavefront.  On curved meshes faces tilt, so the quadrant order no longer
// follows the flow, and a face can be inflow at some points and outflow at others,
// which couples the two elements both ways (the lagging situation the paper describes
// for re-entrant faces in its thick-diffusion section).  The graph's strongly
// connected components ("groups") are solved as units; everything else is a DAG
// processed level by level.  A group is solved directly from a small dense system for
// the traces its members exchange (its inverse is formed by the factorisation), or,
// beyond the direct size limits, by an inner block Gauss-Seidel iteration for which the
// members are ordered along the net face flux so that only the minority points of
// mixed faces are iterated.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <thread>

#include "common.h"

namespace vef {

namespace {

struct DirGraph {
  std::vector<int> comp;          // [E] component id
  std::vector<int> comp_level;    // [ncomp]
  std::vector<int> comp_first;    // [ncomp+1] offsets into comp_members
  std::vector<int> comp_members;  // ordered members
  std::vector<uint16_t> info;     // [E] face bits
  int ncomp = 0;
  int levels = 0;
  long long lagged = 0;
  long long groups = 0;
};

inline int nb_of(int nx, int ny, int e, int f) {
  int i = e % nx, j = e / nx;
  switch (f) {
    case 0: return j > 0 ? e - nx : -1;
    case 1: return i < nx - 1 ? e + 1 : -1;
    case 2: return j < ny - 1 ? e + nx : -1;
    default: return i > 0 ? e - 1 : -1;
  }
}
constexpr int kOpp[4] = {2, 3, 0, 1};

// What the schedule of one direction depends on: the structured mesh's sizes, the outward
// n ds at the face Gauss points ([E][4][nq][2], host copy) and the Gauss weights.
struct HostGeom {
  int nx, ny, nq;
  const double* nds;
  const double* glw;
};

void build_direction(const HostGeom& M, double mu, double eta, DirGraph& G) {
  const int nx = M.nx, ny = M.ny, nq = M.nq;
  const int E = nx * ny;
  const double* nds = M.nds;
  G.info.assign(E, 0);
  // face signs
  for (int e = 0; e < E; ++e) {
    uint16_t bits = 0;
    for (int f = 0; f < 4; ++f) {
      bool anyin = false, anyout = false;
      for (int k = 0; k < nq; ++k) {
        const double* v = nds + (((size_t)e * 4 + f) * nq + k) * 2;
        double s = mu * v[0] + eta * v[1];
        if (s < 0.0) anyin = true;
        if (s > 0.0) anyout = true;
      }
      const int nb = nb_of(nx, ny, e, f);
      if (anyin) bits |= (uint16_t)(1u << f);
      if (anyout && nb >= 0) bits |= (uint16_t)(1u << (8 + f));
    }
    G.info[e] = bits;
  }
  // Tarjan's strongly connected components, iterative.  Edges: donor -> receiver, i.e.
  // from e to its neighbour across f when bit 8+f (neighbour has inflow from e).
  std::vector<int> index(E, -1), low(E, 0), stack;
  std::vector<char> onstack(E, 0);
  G.comp.assign(E, -1);
  stack.reserve(1024);
  int idx = 0, ncomp = 0;
  std::vector<std::pair<int, int>> call;  // (node, next face)
  for (int s = 0; s < E; ++s) {
    if (index[s] >= 0) continue;
    call.push_back({s, 0});
    index[s] = low[s] = idx++;
    stack.push_back(s);
    onstack[s] = 1;
    while (!call.empty()) {
      int v = call.back().first;
      int& f = call.back().second;
      if (f < 4) {
        int ff = f++;
        if (!(G.info[v] & (1u << (8 + ff)))) continue;
        int w = nb_of(nx, ny, v, ff);
        if (index[w] < 0) {
          index[w] = low[w] = idx++;
          stack.push_back(w);
          onstack[w] = 1;
          call.push_back({w, 0});
        } else if (onstack[w]) {
          low[v] = std::min(low[v], index[w]);
        }
        continue;
      }
      if (low[v] == index[v]) {
        int w;
        do {
          w = stack.back();
          stack.pop_back();
          onstack[w] = 0;
          G.comp[w] = ncomp;
        } while (w != v);
        ++ncomp;
      }
      call.pop_back();
      if (!call.empty()) {
        int u = call.back().first;
        low[u] = std::min(low[u], low[v]);
      }
    }
  }
  G.ncomp = ncomp;
  // members per component
  std::vector<int> csize(ncomp, 0);
  for (int e = 0; e < E; ++e) csize[G.comp[e]]++;
  G.comp_first.assign(ncomp + 1, 0);
  for (int c = 0; c < ncomp; ++c) G.comp_first[c + 1] = G.comp_first[c] + csize[c];
  G.comp_members.assign(E, 0);
  {
    std::vector<int> fill(G.comp_first.begin(), G.comp_first.end() - 1);
    for (int e = 0; e < E; ++e) G.comp_members[fill[G.comp[e]]++] = e;
  }
  const int sx = mu >= 0 ? 1 : -1, sy = eta >= 0 ? 1 : -1;
  auto qkey = [&](int e) {
    int i = e % nx, j = e / nx;
    return (sx > 0 ? i : nx - 1 - i) + (sy > 0 ? j : ny - 1 - j);
  };
  // order members of multi-element groups along the net face flux; set intra bits
  for (int c = 0; c < ncomp; ++c) {
    int b = G.comp_first[c], n = csize[c];
    if (n == 1) continue;
    G.groups++;
    std::vector<int> mem(G.comp_members.begin() + b, G.comp_members.begin() + b + n);
    std::vector<int> indeg(n, 0);
    std::vector<std::vector<int>> out(n);
    auto pos = [&](int e) { return (int)(std::find(mem.begin(), mem.end(), e) - mem.begin()); };
    for (int a = 0; a < n; ++a) {
      int u = mem[a];
      for (int f = 0; f < 4; ++f) {
        int w = nb_of(nx, ny, u, f);
        if (w < 0 || G.comp[w] != c) continue;
        G.info[u] |= (uint16_t)(1u << (4 + f));
        double net = 0.0;
        for (int k = 0; k < nq; ++k) {
          const double* v = nds + (((size_t)u * 4 + f) * nq + k) * 2;
          double s = mu * v[0] + eta * v[1];
          net += M.glw[k] * s;
          if (s < 0.0) G.lagged++;
        }
        if (net > 0.0) {  // u feeds w on balance
          out[a].push_back(pos(w));
          indeg[pos(w)]++;
        }
      }
    }
    std::vector<int> order;
    std::vector<char> done(n, 0);
    for (int it = 0; it < n; ++it) {
      int best = -1;
      for (int a = 0; a < n; ++a) {
        if (done[a]) continue;
        if (best < 0 || indeg[a] < indeg[best] ||
            (indeg[a] == indeg[best] && qkey(mem[a]) < qkey(mem[best])))
          best = a;
      }
      done[best] = 1;
      order.push_back(mem[best]);
      for (int w : out[best]) indeg[w]--;
    }
    std::copy(order.begin(), order.end(), G.comp_members.begin() + b);
  }
  // levels of the condensed DAG (Kahn)
  std::vector<int> cindeg(ncomp, 0);
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 4; ++f)
      if (G.info[e] & (1u << (8 + f))) {
        int w = nb_of(nx, ny, e, f);
        if (G.comp[w] != G.comp[e]) cindeg[G.comp[w]]++;
      }
  G.comp_level.assign(ncomp, 0);
  std::vector<int> queue;
  queue.reserve(ncomp);
  for (int c = 0; c < ncomp; ++c)
    if (cindeg[c] == 0) queue.push_back(c);
  size_t head = 0;
  int maxl = 0;
  while (head < queue.size()) {
    int c = queue[head++];
    maxl = std::max(maxl, G.comp_level[c]);
    for (int t = G.comp_first[c]; t < G.comp_first[c + 1]; ++t) {
      int e = G.comp_members[t];
      for (int f = 0; f < 4; ++f) {
        if (!(G.info[e] & (1u << (8 + f)))) continue;
        int w = nb_of(nx, ny, e, f);
        int cw = G.comp[w];
        if (cw == c) continue;
        G.comp_level[cw] = std::max(G.comp_level[cw], G.comp_level[c] + 1);
        if (--cindeg[cw] == 0) queue.push_back(cw);
      }
    }
  }
  G.levels = maxl + 1;
}

template <typename T>
vef_status upload(T** dst, const std::vector<T>& src) {
  VEF_CUDA_TRY(cudaMalloc((void**)dst, std::max<size_t>(1, src.size()) * sizeof(T)));
  if (!src.empty())
    VEF_CUDA_TRY(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return VEF_OK;
}

}  // namespace

Schedule* get_schedule(Mesh* mesh, const double* omega, const double* weights, int D,
                       cudaStream_t stream, vef_status* st) {
  *st = VEF_OK;
  for (auto& s : mesh->schedules) {
    if (s->D == D && std::memcmp(s->omega.data(), omega, sizeof(double) * 2 * D) == 0 &&
        std::memcmp(s->weights.data(), weights, sizeof(double) * D) == 0)
      return s.get();
  }
  const Mesh& M = *mesh;
  const int E = (int)M.E;
  const HostGeom H{M.nx, M.ny, M.nq, M.nds_host.data(), M.tab.glw};
  std::vector<DirGraph> graphs(D);
  {
    unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 32));
    nt = std::min<unsigned>(nt, (unsigned)D);
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t)
      pool.emplace_back([&, t]() {
        for (int d = (int)t; d < D; d += (int)nt)
          build_direction(H, omega[2 * d], omega[2 * d + 1], graphs[d]);
      });
    for (auto& th : pool) th.join();
  }
  std::unique_ptr<Schedule> S(new Schedule());
  S->D = D;
  S->omega.assign(omega, omega + 2 * D);
  S->weights.assign(weights, weights + D);
  S->members = (long long)D * E;
  int levels = 0;
  for (auto& g : graphs) {
    levels = std::max(levels, g.levels);
    S->coupled_groups += g.groups;
    S->lagged_points += g.lagged;
  }
  S->levels = levels;
  // Per direction, its levels in order; inside a level the single-element tasks first,
  // then the coupled groups.  Slots, members and factor records all follow this order.
  std::vector<int> dir_lev0(D + 1, 0), lev_begin, lev_gbegin, lev_mbegin, slot_first, slot_count;
  std::vector<uint32_t> member_code;
  std::vector<int> member_of((size_t)D * E, -1);
  std::vector<int> level_of((size_t)D * E, -1);
  member_code.reserve((size_t)D * E);
  auto add_member = [&](int d, int e, int L) {
    member_of[(size_t)d * E + e] = (int)member_code.size();
    level_of[(size_t)d * E + e] = L;
    member_code.push_back(((uint32_t)d << 22) | (uint32_t)e);
  };
  for (int d = 0; d < D; ++d) {
    const DirGraph& g = graphs[d];
    dir_lev0[d] = (int)lev_begin.size();
    std::vector<std::vector<int>> bylevel(g.levels);
    for (int c = 0; c < g.ncomp; ++c) bylevel[g.comp_level[c]].push_back(c);
    for (int L = 0; L < g.levels; ++L) {
      lev_begin.push_back((int)slot_first.size());
      lev_mbegin.push_back((int)member_code.size());
      for (int c : bylevel[L]) {
        const int b = g.comp_first[c], n = g.comp_first[c + 1] - b;
        if (n != 1) continue;
        slot_first.push_back((int)member_code.size());
        slot_count.push_back(1);
        add_member(d, g.comp_members[b], L);
      }
      lev_gbegin.push_back((int)slot_first.size());
      for (int c : bylevel[L]) {
        const int b = g.comp_first[c], n = g.comp_first[c + 1] - b;
        if (n == 1) continue;
        slot_first.push_back((int)member_code.size());
        slot_count.push_back(n);
        for (int t = 0; t < n; ++t) add_member(d, g.comp_members[b + t], L);
      }
    }
  }
  dir_lev0[D] = (int)lev_begin.size();
  lev_begin.push_back((int)slot_first.size());
  S->total_levels = dir_lev0[D];
  // Validate the order the sweep relies on: every element is scheduled once, and each
  // external upwind donor sits at an earlier level of the same direction.
  for (size_t t = 0; t < member_of.size(); ++t)
    if (member_of[t] < 0) {
      set_last_error("internal error: sweep schedule misses an element");
      *st = VEF_ERR_INVALID_ARG;
      return nullptr;
    }
  for (int d = 0; d < D; ++d)
    for (int e = 0; e < E; ++e) {
      const uint16_t bits = graphs[d].info[e];
      for (int f = 0; f < 4; ++f) {
        if (!(bits & (1u << f)) || (bits & (1u << (4 + f)))) continue;
        const int nb = nb_of(M.nx, M.ny, e, f);
        if (nb < 0) continue;
        if (level_of[(size_t)d * E + nb] >= level_of[(size_t)d * E + e]) {
          set_last_error("internal error: sweep schedule violates the dependency order");
          *st = VEF_ERR_INVALID_ARG;
          return nullptr;
        }
      }
    }
  S->nslots = (long long)slot_first.size();

  std::vector<uint16_t> faceinfo((size_t)D * E);
  for (int d = 0; d < D; ++d)
    std::copy(graphs[d].info.begin(), graphs[d].info.end(), faceinfo.begin() + (size_t)d * E);
  std::vector<double> om(omega, omega + 2 * D), wt(weights, weights + D);
  if ((*st = upload(&S->dir_lev0, dir_lev0)) != VEF_OK) return nullptr;
  if ((*st = upload(&S->lev_begin, lev_begin)) != VEF_OK) return nullptr;
  if ((*st = upload(&S->lev_gbegin, lev_gbegin)) != VEF_OK) return nullptr;
  if ((*st = upload(&S->lev_mbegin, lev_mbegin)) != VEF_OK) return nullptr;
  {
    std::vector<uint2> minfo(member_code.size());
    for (size_t m = 0; m < member_code.size(); ++m) {
      const int d = (int)(member_code[m] >> 22), e = (int)(member_code[m] & ((1u << 22) - 1));
      minfo[m] = make_uint2((unsigned)e, (unsigned)graphs[d].info[e]);
    }
    if ((*st = upload(&S->member_info, minfo)) != VEF_OK) return nullptr;
    // byte f of member_nbpos: position inside the member's group of its neighbour across
    // face f when that neighbour is in the same group, else 255
    std::vector<uint32_t> nbpos(member_code.size(), 0xffffffffu);
    for (size_t sl = 0; sl < slot_first.size(); ++sl) {
      if (slot_count[sl] == 1) continue;
      const int first = slot_first[sl], cnt = slot_count[sl];
      for (int t = 0; t < cnt; ++t) {
        const int m = first + t;
        const int d = (int)(member_code[m] >> 22), e = (int)(member_code[m] & ((1u << 22) - 1));
        uint32_t packed = 0xffffffffu;
        for (int f = 0; f < 4; ++f) {
          if (!(graphs[d].info[e] & (1u << (4 + f)))) continue;
          const int pos = member_of[(size_t)d * E + nb_of(M.nx, M.ny, e, f)] - first;
          if (pos >= 0 && pos < 255) packed = (packed & ~(0xffu << (8 * f))) | ((uint32_t)pos << (8 * f));
        }
        nbpos[m] = packed;
      }
    }
    if ((*st = upload(&S->member_nbpos, nbpos)) != VEF_OK) return nullptr;
  }
  // Coupled groups solved directly.  For member a (in group order) and face f that is
  // inflow somewhere and shared with another member b, the Q values of b's trace on that
  // face are trace unknowns, numbered by member, then face, then face node.  Groups with
  // more members or unknowns than the direct limits keep slot_gid = -1.
  {
    const int Q = M.p + 1;
    std::vector<int> slot_gid(slot_first.size(), -1), grp_slot, grp_nt;
    std::vector<long long> grp_toff(1, 0);
    std::vector<std::pair<int, int>> direct;   // (nt, slot)
    for (size_t sl = 0; sl < slot_first.size(); ++sl) {
      const int cnt = slot_count[sl];
      if (cnt == 1 || cnt > group_direct_members(M.p)) continue;
      int couplings = 0;
      for (int t = 0; t < cnt; ++t) {
        const uint32_t code = member_code[slot_first[sl] + t];
        const uint16_t bits = graphs[code >> 22].info[code & ((1u << 22) - 1)];
        for (int f = 0; f < 4; ++f)
          if ((bits & (1u << f)) && (bits & (1u << (4 + f)))) ++couplings;
      }
      const int nt = couplings * Q;
      if (nt == 0 || nt > kGroupMaxTrace) continue;
      direct.push_back({nt, (int)sl});
    }
    // groups numbered by size, so the factorisation can give the small trace systems
    // (the great majority) a launch with little shared memory per CTA
    std::stable_sort(direct.begin(), direct.end(),
                     [](const std::pair<int, int>& x, const std::pair<int, int>& y) { return x.first < y.first; });
    for (const auto& g : direct) {
      slot_gid[g.second] = (int)grp_slot.size();
      grp_slot.push_back(g.second);
      grp_nt.push_back(g.first);
      // offsets rounded to 4 entries keep every inverse 16-byte aligned in both precisions
      grp_toff.push_back(grp_toff.back() + ((long long)g.first * g.first + 3) / 4 * 4);
      S->max_nt = std::max(S->max_nt, g.first);
      for (int b = 0; b < 3; ++b)
        if (g.first <= (8 << b)) ++S->ngroups_upto[b];
    }
    S->ngroups = (long long)grp_slot.size();
    S->grec_elems = grp_toff.back();
    if ((*st = upload(&S->slot_gid, slot_gid)) != VEF_OK) return nullptr;
    if ((*st = upload(&S->grp_slot, grp_slot)) != VEF_OK) return nullptr;
    if ((*st = upload(&S->grp_nt, grp_nt)) != VEF_OK) return nullptr;
    if ((*st = upload(&S->grp_toff, grp_toff)) != VEF_OK) return nullptr;
  }
  // Shared-memory trace slots of the single-CTA sweep (two reserved, see kTraceZero).
  // Per direction, levels in order: a
  // single-element task that feeds a later single-element task across a face takes a free
  // slot for that face's node values, released once the receiver's level is done, so a
  // slot freed at level L is reused from level L + 1 on (reads and writes of one level
  // never share a slot).  Receivers whose face is not one of their two staged W slots,
  // coupled-group members and couplings beyond the capacity keep 0xffff: the receiver
  // reads the donor's psi from global memory instead.
  {
    int cap = cta_trace_capacity(M.p);
    if (const char* env = std::getenv("VEF_TRACE_SLOTS")) cap = std::max(0, std::min(cap, std::atoi(env)));
    const unsigned zz = kTraceZero | (kTraceZero << 16), ss = kTraceSink | (kTraceSink << 16);
    std::vector<uint4> tslot(member_code.size(), make_uint4(zz, ss, ss, 0u));
    std::vector<int> dir_live(D, 0);
    std::vector<long long> dir_global(D, 0);
    auto set16 = [](unsigned& w, int half, unsigned id) {
      w = (w & ~(0xffffu << (16 * half))) | (id << (16 * half));
    };
    auto interior_inflow_rank = [&](int d, int e, int g) {
      const uint16_t bits = graphs[d].info[e];
      int r = 0;
      for (int f = 0; f < g; ++f)
        if ((bits & (1u << f)) && nb_of(M.nx, M.ny, e, f) >= 0) ++r;
      return r;
    };
    auto run = [&](int d) {
      const DirGraph& g = graphs[d];
      std::vector<unsigned> free_ids;
      free_ids.reserve(cap);
      for (int id = cap - 1; id >= (int)kTraceFirst; --id) free_ids.push_back((unsigned)id);
      std::vector<std::vector<unsigned>> release(g.levels);
      int live = (int)kTraceFirst;
      dir_live[d] = live;
      for (int L = 0; L < g.levels; ++L) {
        const int k = dir_lev0[d] + L;
        const int m0 = lev_mbegin[k];
        const int nsingle = lev_gbegin[k] - lev_begin[k];
        for (int m = m0; m < m0 + nsingle; ++m) {
          const int e = (int)(member_code[m] & ((1u << 22) - 1));
          const uint16_t bits = g.info[e];
          for (int f = 0; f < 4; ++f) {
            if (!(bits & (1u << (8 + f)))) continue;
            const int w = nb_of(M.nx, M.ny, e, f);
            const int wm = member_of[(size_t)d * E + w];
            const int Lw = level_of[(size_t)d * E + w];
            const int kw = dir_lev0[d] + Lw;
            if (wm >= lev_mbegin[kw] + (lev_gbegin[kw] - lev_begin[kw])) continue;  // group member
            const int rank = interior_inflow_rank(d, w, kOpp[f]);
            if (rank >= 2) continue;
            if (free_ids.empty()) { ++dir_global[d]; continue; }
            const unsigned id = free_ids.back();
            free_ids.pop_back();
            set16(f < 2 ? tslot[m].y : tslot[m].z, f & 1, id);
            set16(tslot[wm].x, rank, id);
            release[Lw].push_back(id);
            dir_live[d] = std::max(dir_live[d], ++live);
          }
        }
        for (unsigned id : release[L]) free_ids.push_back(id);
        live -= (int)release[L].size();
        std::vector<unsigned>().swap(release[L]);
      }
      // members whose couplings are not all in shared memory.  Bit 0 (forward sweep): an
      // interior inflow face beyond the two staged W slots, or a staged one left without a
      // slot.  Bit 1 (adjoint sweep, where the receivers write and the donors read the same
      // slots): a face toward a receiver whose slot is missing (kTraceSink).
      for (int L = 0; L < g.levels; ++L) {
        const int k = dir_lev0[d] + L;
        const int m0 = lev_mbegin[k];
        const int nsingle = lev_gbegin[k] - lev_begin[k];
        for (int m = m0; m < m0 + nsingle; ++m) {
          const int e = (int)(member_code[m] & ((1u << 22) - 1));
          int rank = 0;
          for (int f = 0; f < 4; ++f) {
            if (!(g.info[e] & (1u << f)) || nb_of(M.nx, M.ny, e, f) < 0) continue;
            if (rank >= 2 || ((tslot[m].x >> (16 * rank)) & 0xffffu) == kTraceZero) tslot[m].w |= 1u;
            ++rank;
          }
          for (int f = 0; f < 4; ++f) {
            if (!(g.info[e] & (1u << (8 + f)))) continue;
            const unsigned wid = ((f < 2 ? tslot[m].y : tslot[m].z) >> (16 * (f & 1))) & 0xffffu;
            if (wid == kTraceSink) tslot[m].w |= 2u;
          }
        }
      }
    };
    unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 32));
    nt = std::min<unsigned>(nt, (unsigned)D);
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t)
      pool.emplace_back([&, t]() {
        for (int d = (int)t; d < D; d += (int)nt) run(d);
      });
    for (auto& th : pool) th.join();
    for (int d = 0; d < D; ++d) {
      S->trace_slots = std::max(S->trace_slots, dir_live[d]);
      S->trace_global += dir_global[d];
    }
    if ((*st = upload(&S->tslot, tslot)) != VEF_OK) return nullptr;
  }
  if ((*st = upload(&S->slot_first, slot_first)) != VEF_OK) return nullptr;
  if ((*st = upload(&S->slot_count, slot_count)) != VEF_OK) return nullptr;
  if ((*st = upload(&S->member_code, member_code)) != VEF_OK) return nullptr;
  if ((*st = upload(&S->member_of, member_of)) != VEF_OK) return nullptr;
  if ((*st = upload(&S->faceinfo, faceinfo)) != VEF_OK) return nullptr;
  if ((*st = upload(&S->omega_dev, om)) != VEF_OK) return nullptr;
  if ((*st = upload(&S->weights_dev, wt)) != VEF_OK) return nullptr;
  (void)stream;
  mesh->schedules.push_back(std::move(S));
  return mesh->schedules.back().get();
}

}  // namespace vef

extern "C" vef_status vef_schedule_host(int nx, int ny, int p, const double* nds, const double* omega,
                                        int D, int* levels, long long* groups, int* level,
                                        int* comp_size) {
  using namespace vef;
  if (nx < 1 || ny < 1 || (long long)nx * ny > kMaxE) {
    set_last_error("nx, ny must be >= 1 with nx*ny <= 2^22");
    return VEF_ERR_INVALID_ARG;
  }
  if (p < 1 || p > kMaxP) { set_last_error("p must be in 1..4"); return VEF_ERR_INVALID_ARG; }
  if (D < 1 || D > kMaxD) { set_last_error("D must be in 1..1023"); return VEF_ERR_INVALID_ARG; }
  if (!nds || !omega || !levels || !groups) {
    set_last_error("nds, omega, levels and groups are required");
    return VEF_ERR_INVALID_ARG;
  }
  try {
    const Tab1D tab = make_tab1d(p);
    const HostGeom H{nx, ny, p + 2, nds, tab.glw};
    const size_t E = (size_t)nx * ny;
    for (int d = 0; d < D; ++d) {
      DirGraph G;
      build_direction(H, omega[2 * d], omega[2 * d + 1], G);
      levels[d] = G.levels;
      groups[d] = G.groups;
      for (size_t e = 0; e < E; ++e) {
        const int c = G.comp[e];
        if (level) level[d * E + e] = G.comp_level[c];
        if (comp_size) comp_size[d * E + e] = G.comp_first[c + 1] - G.comp_first[c];
      }
    }
  } catch (const std::bad_alloc&) {
    set_last_error("out of host memory");
    return VEF_ERR_OOM;
  }
  return VEF_OK;
}
