// Host side of the library: parameters, error strings and the graph plan --
// pool offsets, work tiles, and the symbolic block Cholesky of every graph's
// gauge-reduced 7N system (Sec. 3.5: "sparse Cholesky decomposition as the
// system is not dense"), ordered by greedy minimum degree.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <memory>
#include <set>
#include <vector>

#include "common.cuh"

struct mslam_plan {
  int32_t N = 0, E = 0, G = 0;
  std::vector<int32_t> kf_hw, edges, graph_of_kf;
  std::vector<int64_t> kf_off, e_off;
  std::vector<mslam::DevEdge> dedges;
  std::vector<mslam::DevTile> tiles;
  std::vector<mslam::DevGraph> graphs;
  std::vector<int32_t> ints;
  std::vector<int32_t> order;
  int64_t n_blocks_total = 0, n_trips_total = 0, solve_ws_doubles = 0, max_graph_doubles = 0;
  int64_t max_mixed_bytes = 0;  // shared memory of the mixed-precision solve for the largest graph
  int64_t max_mixed_bytes_nofactor = 0;  // the same with the FP32 factor left in the workspace
  int64_t max_mixed_elems = 0;  // elements its assembly kernel covers for the largest graph
  int32_t max_m = 0;            // non-fixed poses of the largest graph
  int32_t max_levels = 0;
  int32_t lin_tile = 0, lin_blocks_per_sm = 0, match_bx = 0, match_by = 0, lin_form = 0, solve_form = 0;
  int32_t wait_limit = 0, match_form = 0, match_ppt = 1;
  int32_t n_mblocks = 0;
  void* dev = nullptr;
  size_t dev_bytes = 0;
  size_t off_edges = 0, off_tiles = 0, off_graphs = 0, off_ints = 0, blob_bytes = 0;
};

namespace mslam {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

mslam_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MSLAM_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return MSLAM_ERR_CUDA;
}

bool check_plan_uploaded(const mslam_plan* plan) {
  if (!plan) {
    set_error("plan is NULL");
    return false;
  }
  if (!plan->dev) {
    set_error("plan has not been uploaded (mslam_plan_upload)");
    return false;
  }
  return true;
}

PlanView plan_view(const mslam_plan* plan) {
  PlanView v;
  const char* base = static_cast<const char*>(plan->dev);
  v.N = plan->N;
  v.E = plan->E;
  v.G = plan->G;
  v.n_tiles = (int32_t)plan->tiles.size();
  v.n_mblocks = plan->n_mblocks;
  v.P = plan->e_off.back();
  v.lin_tile = plan->lin_tile;
  v.match_bx = plan->match_bx;
  v.match_by = plan->match_by;
  v.match_ppt = plan->match_ppt;
  v.wait_polls = plan->wait_limit < 0 ? 0u : plan->wait_limit == 0 ? (1u << 24) : (uint32_t)plan->wait_limit;
  v.edges = reinterpret_cast<const DevEdge*>(base + plan->off_edges);
  v.tiles = reinterpret_cast<const DevTile*>(base + plan->off_tiles);
  v.graphs = reinterpret_cast<const DevGraph*>(base + plan->off_graphs);
  v.ints = reinterpret_cast<const int32_t*>(base + plan->off_ints);
  return v;
}

void plan_edge_tiles(const mslam_plan* plan, int e, int* t0, int* t1) {
  *t0 = plan->dedges[e].tile_begin;
  *t1 = plan->dedges[e].tile_end;
}

void plan_edge_mblocks(const mslam_plan* plan, int e, int* b0, int* b1) {
  *b0 = plan->dedges[e].mblock_begin;
  *b1 = (e + 1 < plan->E) ? plan->dedges[e + 1].mblock_begin : plan->n_mblocks;
}

int64_t plan_max_graph_doubles(const mslam_plan* plan) { return plan->max_graph_doubles; }
int64_t plan_max_mixed_bytes(const mslam_plan* plan) { return plan->max_mixed_bytes; }
int64_t plan_max_mixed_bytes_nofactor(const mslam_plan* plan) { return plan->max_mixed_bytes_nofactor; }
bool plan_tracking_form(const mslam_plan* plan) {
  if (plan->E == 0 || plan->E != plan->G) return false;
  std::vector<int> per_graph(plan->G, 0);
  for (const auto& e : plan->dedges) ++per_graph[e.graph];
  for (int g = 0; g < plan->G; ++g)
    if (per_graph[g] != 1 || plan->graphs[g].m != 1) return false;
  return true;
}
int64_t plan_max_mixed_elems(const mslam_plan* plan) { return plan->max_mixed_elems; }
int plan_max_unknown_blocks(const mslam_plan* plan) { return plan->max_m; }
int64_t plan_solve_ws_doubles(const mslam_plan* plan) { return plan->solve_ws_doubles; }
int plan_lin_blocks_per_sm(const mslam_plan* plan) { return plan->lin_blocks_per_sm; }
int plan_lin_form(const mslam_plan* plan) { return plan->lin_form; }
int plan_solve_form(const mslam_plan* plan) { return plan->solve_form; }
int plan_match_form(const mslam_plan* plan) { return plan->match_form; }
int64_t plan_edge_off(const mslam_plan* plan, int e) { return plan->e_off[e]; }
int plan_max_image_dim(const mslam_plan* plan) {
  int m = 0;
  for (int v : plan->kf_hw) m = std::max(m, v);
  return m;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Symbolic factorisation of one graph.
static void build_graph(mslam_plan* P, int g, const std::vector<int>& kfs) {
  DevGraph dg{};
  const int gauge = kfs.front();  // lowest-indexed keyframe of the graph
  dg.gauge = gauge;
  const int m = (int)kfs.size() - 1;
  dg.m = m;
  // undirected adjacency between the non-fixed keyframes
  std::map<int, std::set<int>> adj;
  for (int k : kfs)
    if (k != gauge) adj[k];
  for (int e = 0; e < P->E; ++e) {
    const int i = P->edges[2 * e], j = P->edges[2 * e + 1];
    if (P->graph_of_kf[i] != g) continue;
    if (i != gauge && j != gauge) {
      adj[i].insert(j);
      adj[j].insert(i);
    }
  }
  // greedy minimum degree (ties: lowest keyframe index); elimination makes
  // the remaining neighbours a clique, whose members become column rows
  std::vector<int> pos_kf;          // elimination position -> keyframe
  std::vector<std::vector<int>> nb; // neighbours (keyframes) at elimination
  std::map<int, std::set<int>> live = adj;
  while (!live.empty()) {
    int best = -1;
    size_t bd = SIZE_MAX;
    for (auto& kv : live)
      if (kv.second.size() < bd) {
        bd = kv.second.size();
        best = kv.first;
      }
    std::vector<int> ns(live[best].begin(), live[best].end());
    for (int a : ns) {
      live[a].erase(best);
      for (int b : ns)
        if (a != b) live[a].insert(b);
    }
    live.erase(best);
    pos_kf.push_back(best);
    nb.push_back(ns);
  }
  std::map<int, int> pos_of;
  for (int p = 0; p < m; ++p) pos_of[pos_kf[p]] = p;
  for (int p = 0; p < m; ++p) P->order[pos_kf[p]] = p;
  P->order[gauge] = -1;

  // L pattern: column p has rows pos_of[neighbours] (all > p), sorted
  std::vector<std::vector<int>> rows(m);
  for (int p = 0; p < m; ++p) {
    for (int k : nb[p]) rows[p].push_back(pos_of[k]);
    std::sort(rows[p].begin(), rows[p].end());
  }
  std::map<std::pair<int, int>, int> blk;  // (row, col) -> block id
  int nb_total = m;
  for (int p = 0; p < m; ++p)
    for (int r : rows[p]) blk[{r, p}] = nb_total++;
  dg.n_blocks = nb_total;

  std::vector<int32_t>& I = P->ints;
  dg.off_pose = (int32_t)I.size();
  for (int p = 0; p < m; ++p) I.push_back(pos_kf[p]);
  dg.off_col = (int32_t)I.size();
  {
    int acc = 0;
    for (int p = 0; p <= m; ++p) {
      I.push_back(acc);
      if (p < m) acc += (int)rows[p].size();
    }
  }
  dg.off_colent = (int32_t)I.size();
  for (int p = 0; p < m; ++p)
    for (int r : rows[p]) {
      I.push_back(r);
      I.push_back(blk[{r, p}]);
    }
  // update triples of column p: A(rb, ra) -= L(rb, p) L(ra, p)^T for ra <= rb
  dg.off_trip = (int32_t)I.size();
  std::vector<int32_t> trips;
  {
    int acc = 0;
    std::vector<int> ptr;
    for (int p = 0; p < m; ++p) {
      ptr.push_back(acc);
      const auto& R = rows[p];
      for (size_t a = 0; a < R.size(); ++a)
        for (size_t b = a; b < R.size(); ++b) {
          const int ra = R[a], rb = R[b];
          const int target = (ra == rb) ? ra : blk.at({rb, ra});
          trips.push_back(target);
          trips.push_back(blk.at({rb, p}));
          trips.push_back(blk.at({ra, p}));
          ++acc;
        }
    }
    ptr.push_back(acc);
    for (int v : ptr) I.push_back(v);
    P->n_trips_total += acc;
  }
  dg.off_tripent = (int32_t)I.size();
  I.insert(I.end(), trips.begin(), trips.end());

  // ---- level schedule for the left-looking factorisation.  Column p depends
  // on every column c with p in rows(c); lev(p) = 1 + max lev(c).  Columns of
  // one level touch disjoint blocks, so a level is processed in parallel.
  std::vector<int> lev(m, 0);
  int n_lev = 0;
  for (int c = 0; c < m; ++c)
    for (int r : rows[c]) lev[r] = std::max(lev[r], lev[c] + 1);
  for (int c = 0; c < m; ++c) n_lev = std::max(n_lev, lev[c] + 1);
  std::vector<std::vector<int>> cols_of(n_lev);
  for (int c = 0; c < m; ++c) cols_of[lev[c]].push_back(c);
  // update pairs grouped by target block: A_t -= L_b L_a^T in increasing c
  std::vector<std::vector<std::pair<int, int>>> by_target(nb_total);
  std::vector<std::vector<std::pair<int, int>>> rowstruct(m);  // p -> (c, block L(p, c))
  for (int c = 0; c < m; ++c) {
    const auto& R = rows[c];
    for (size_t a = 0; a < R.size(); ++a) {
      rowstruct[R[a]].push_back({c, blk.at({R[a], c})});
      for (size_t b = a; b < R.size(); ++b) {
        const int ra = R[a], rb = R[b];
        const int target = (ra == rb) ? ra : blk.at({rb, ra});
        by_target[target].push_back({blk.at({rb, c}), blk.at({ra, c})});
      }
    }
  }
  dg.n_levels = n_lev;
  dg.off_lev = (int32_t)I.size();  // lev_ptr [n_lev + 1] into lev_cols
  {
    int acc = 0;
    for (int l = 0; l <= n_lev; ++l) {
      I.push_back(acc);
      if (l < n_lev) acc += (int)cols_of[l].size();
    }
  }
  dg.off_levcols = (int32_t)I.size();
  for (auto& v : cols_of) I.insert(I.end(), v.begin(), v.end());
  // per level: target blocks (diagonal then column blocks of each column)
  dg.off_levtgt = (int32_t)I.size();  // [n_lev + 1] pointers into the target list
  std::vector<int32_t> tg_list;
  {
    std::vector<int32_t> ptr;
    for (int l = 0; l < n_lev; ++l) {
      ptr.push_back((int32_t)tg_list.size());
      for (int c : cols_of[l]) {
        tg_list.push_back(c);
        for (int r : rows[c]) tg_list.push_back(blk.at({r, c}));
      }
    }
    ptr.push_back((int32_t)tg_list.size());
    I.insert(I.end(), ptr.begin(), ptr.end());
  }
  dg.off_tgtlist = (int32_t)I.size();
  I.insert(I.end(), tg_list.begin(), tg_list.end());
  dg.off_tptr = (int32_t)I.size();  // [n_blocks + 1] into pairs
  {
    int acc = 0;
    for (int b = 0; b <= nb_total; ++b) {
      I.push_back(acc);
      if (b < nb_total) acc += (int)by_target[b].size();
    }
  }
  dg.off_pairs = (int32_t)I.size();
  for (auto& v : by_target)
    for (auto& pr : v) {
      I.push_back(pr.first);
      I.push_back(pr.second);
    }
  // per level: the targets with at least one update pair (the rest need no update phase)
  dg.off_levupd = (int32_t)I.size();
  {
    std::vector<int32_t> ptr, lst;
    for (int l = 0; l < n_lev; ++l) {
      ptr.push_back((int32_t)lst.size());
      for (int c : cols_of[l]) {
        if (!by_target[c].empty()) lst.push_back(c);
        for (int r : rows[c]) {
          const int t = blk.at({r, c});
          if (!by_target[t].empty()) lst.push_back(t);
        }
      }
    }
    ptr.push_back((int32_t)lst.size());
    I.insert(I.end(), ptr.begin(), ptr.end());
    dg.off_updlist = (int32_t)I.size();
    I.insert(I.end(), lst.begin(), lst.end());
  }
  dg.off_rsptr = (int32_t)I.size();  // [m + 1] row structure (c, block) per position
  {
    int acc = 0;
    for (int q = 0; q <= m; ++q) {
      I.push_back(acc);
      if (q < m) acc += (int)rowstruct[q].size();
    }
  }
  dg.off_rs = (int32_t)I.size();
  for (auto& v : rowstruct)
    for (auto& pr : v) {
      I.push_back(pr.first);
      I.push_back(pr.second);
    }
  dg.off_blkcol = (int32_t)I.size();  // [n_blocks] column position of each block
  for (int b = 0; b < m; ++b) I.push_back(b);
  for (int c = 0; c < m; ++c)
    for (size_t k = 0; k < rows[c].size(); ++k) I.push_back(c);
  P->max_levels = std::max(P->max_levels, n_lev);

  // assembly lists (edge order): quadrant 0 = H_ii, 1 = H_jj, 2 = rows i cols j, 3 = rows j cols i
  std::vector<std::vector<int>> asml(nb_total), gasm(m);
  for (int e = 0; e < P->E; ++e) {
    const int i = P->edges[2 * e], j = P->edges[2 * e + 1];
    if (P->graph_of_kf[i] != g) continue;
    if (i != gauge) {
      asml[pos_of[i]].push_back(4 * e + 0);
      gasm[pos_of[i]].push_back(2 * e + 0);
    }
    if (j != gauge) {
      asml[pos_of[j]].push_back(4 * e + 1);
      gasm[pos_of[j]].push_back(2 * e + 1);
    }
    if (i != gauge && j != gauge) {
      const int pi = pos_of[i], pj = pos_of[j];
      if (pi > pj)
        asml[blk.at({pi, pj})].push_back(4 * e + 2);
      else
        asml[blk.at({pj, pi})].push_back(4 * e + 3);
    }
  }
  dg.off_asm = (int32_t)I.size();
  {
    int acc = 0;
    for (int b = 0; b <= nb_total; ++b) {
      I.push_back(acc);
      if (b < nb_total) acc += (int)asml[b].size();
    }
  }
  dg.off_asment = (int32_t)I.size();
  for (auto& v : asml) I.insert(I.end(), v.begin(), v.end());
  dg.off_gasm = (int32_t)I.size();
  {
    int acc = 0;
    for (int p = 0; p <= m; ++p) {
      I.push_back(acc);
      if (p < m) acc += (int)gasm[p].size();
    }
  }
  dg.off_gasment = (int32_t)I.size();
  for (auto& v : gasm) I.insert(I.end(), v.begin(), v.end());
  dg.int_end = (int32_t)I.size();
  dg.off_blkrow = (int32_t)I.size();  // [n_blocks] row position of each block
  {
    std::vector<int32_t> br(nb_total, 0);
    for (int b = 0; b < m; ++b) br[b] = b;
    for (int p = 0; p < m; ++p)
      for (int r : rows[p]) br[blk[{r, p}]] = r;
    I.insert(I.end(), br.begin(), br.end());
  }

  dg.ws_off = P->solve_ws_doubles;
  // numeric workspace: blocks (49 each), rhs (7 m), assembled diagonal (7 m),
  // reciprocal pivots (7 m)
  const int64_t need = (int64_t)nb_total * 49 + 21 * (int64_t)m;
  P->solve_ws_doubles += need;
  P->max_graph_doubles = std::max(P->max_graph_doubles, need);
  // inputs of the mixed-precision solve, written by its assembly kernel:
  // the scaled FP32 factor (7 x kLfRow floats per block), S and -g
  P->solve_ws_doubles = (P->solve_ws_doubles + 3) & ~int64_t(3);  // 32-byte aligned for vector loads
  dg.ws_mixed = P->solve_ws_doubles;
  P->solve_ws_doubles += (int64_t)nb_total * (7 * kLfRow / 2) + 14 * (int64_t)m;
  // its shared memory: S, x, -g (FP64), the padded FP32 factor, y,
  // pivots and the inverses of the diagonal factor blocks (7 x 8 floats per
  // block column), and the graph's tables except the update triples
  const int64_t table_ints = (int64_t)(dg.off_trip - dg.off_pose) + (int64_t)(dg.int_end - dg.off_lev);
  P->max_mixed_bytes = std::max(P->max_mixed_bytes,
                                (int64_t)(64 * 7 * (int64_t)m + 4 * 7 * kLfRow * (int64_t)nb_total + 4 * table_ints + 16));
  P->max_mixed_bytes_nofactor = std::max(P->max_mixed_bytes_nofactor,
                                         (int64_t)(64 * 7 * (int64_t)m + 4 * table_ints + 16));
  P->max_mixed_elems = std::max(P->max_mixed_elems, (int64_t)nb_total * 7 * kLfRow);
  P->max_m = std::max(P->max_m, (int32_t)m);
  P->n_blocks_total += nb_total;
  P->graphs.push_back(dg);
}

}  // namespace mslam

using namespace mslam;

extern "C" {

void mslam_default_params(mslam_params* p) {
  if (!p) return;
  p->sigma_ray = 0.01f;
  p->sigma_dist = 0.1f;
  p->huber_delta = 1.345f;
  p->q_min = 1.5f;
  p->lm_lambda = 1e-8f;
  p->lm_iters = 10;
  p->win_radius = 3;
  p->n_levels = 2;
  p->win_dilation[0] = 2;
  p->win_dilation[1] = 1;
  p->win_dilation[2] = 1;
  p->win_dilation[3] = 1;
  p->max_rel_dist3d = 0.1f;
  p->conv_tol = 1e-10;
  p->residual = MSLAM_RES_RAY;
  p->sigma_point = 0.05f;
  p->sigma_pixel = 1.0f;
  p->sigma_depth = 0.1f;
  p->fx = p->fy = p->cx = p->cy = 0.0f;
}

const char* mslam_last_error(void) { return g_err; }

const char* mslam_version(void) { return "mslam-gb300 0.1 (sm_103a)"; }

void mslam_default_plan_opts(mslam_plan_opts* o) {
  if (!o) return;
  o->lin_tile = kLinTile;
  o->lin_blocks_per_sm = 0;
  o->match_block_w = kMatchBX;
  o->lin_form = 3;
  o->solve_form = 0;
  o->wait_limit = 0;
  o->match_form = 0;
  o->match_ppt = 1;
}

mslam_status mslam_plan_create(int32_t N, const int32_t* kf_hw, int32_t E, const int32_t* edges,
                               const int32_t* graph_of_kf, mslam_plan** out) {
  return mslam_plan_create_ex(N, kf_hw, E, edges, graph_of_kf, nullptr, out);
}

mslam_status mslam_plan_create_ex(int32_t N, const int32_t* kf_hw, int32_t E, const int32_t* edges,
                                  const int32_t* graph_of_kf, const mslam_plan_opts* opts, mslam_plan** out) {
  mslam_plan_opts o;
  mslam_default_plan_opts(&o);
  if (opts) o = *opts;
  if (o.lin_tile < 1024 || o.lin_tile > 65536 || (o.lin_tile % kLinThreads) != 0 || o.lin_blocks_per_sm < 0 ||
      o.lin_blocks_per_sm > 32 ||
      (o.match_block_w != 4 && o.match_block_w != 8 && o.match_block_w != 16 && o.match_block_w != 32 &&
       o.match_block_w != 64 && o.match_block_w != 128 && o.match_block_w != 256) ||
      o.lin_form < 0 || o.lin_form > 3 || (o.solve_form != 0 && o.solve_form != 1) ||
      (o.match_form < 0 || o.match_form > 2) || o.match_ppt < 1 || o.match_ppt > 2) {
    set_error("plan options: lin_tile %d (multiple of %d in [1024, 65536]), lin_blocks_per_sm %d (0..32), "
              "match_block_w %d (4, 8, ..., 256), lin_form %d (0..3), solve_form %d (0 or 1), match_form %d "
              "(0, 1 or 2), match_ppt %d (1 or 2)", o.lin_tile, kLinThreads, o.lin_blocks_per_sm, o.match_block_w,
              o.lin_form, o.solve_form, o.match_form, o.match_ppt);
    if (out) *out = nullptr;
    return MSLAM_ERR_ARG;
  }
  if (!out) {
    set_error("out is NULL");
    return MSLAM_ERR_ARG;
  }
  *out = nullptr;
  if (N < 1 || !kf_hw || E < 0 || (E > 0 && !edges)) {
    set_error("bad sizes or NULL host arrays (N=%d, E=%d)", N, E);
    return MSLAM_ERR_ARG;
  }
  try {
    // the plan's host tables: an allocation failure returns a status instead
    // of unwinding through the C interface
    std::unique_ptr<mslam_plan> P(new mslam_plan());
    P->lin_tile = o.lin_tile;
    P->lin_blocks_per_sm = o.lin_blocks_per_sm;
    P->lin_form = o.lin_form;
    P->solve_form = o.solve_form;
    P->wait_limit = o.wait_limit;
    P->match_form = o.match_form;
    P->match_ppt = o.match_ppt;
    P->match_bx = o.match_block_w;
    P->match_by = kMatchThreads / o.match_block_w;
    P->N = N;
    P->E = E;
    P->kf_hw.assign(kf_hw, kf_hw + 2 * N);
    P->edges.assign(edges, edges + 2 * (size_t)E);
    P->graph_of_kf.assign(N, 0);
    if (graph_of_kf) P->graph_of_kf.assign(graph_of_kf, graph_of_kf + N);
    int G = 0;
    for (int k = 0; k < N; ++k) {
      const int H = kf_hw[2 * k], W = kf_hw[2 * k + 1];
      if (H < 2 || W < 2 || H > 8192 || W > 8192 || P->graph_of_kf[k] < 0 || P->graph_of_kf[k] >= N) {
        set_error("keyframe %d: bad size %dx%d or graph id %d", k, H, W, P->graph_of_kf[k]);
        return MSLAM_ERR_ARG;
      }
      G = std::max(G, P->graph_of_kf[k] + 1);
    }
    std::vector<std::vector<int>> kfs(G);
    for (int k = 0; k < N; ++k) kfs[P->graph_of_kf[k]].push_back(k);
    for (int g = 0; g < G; ++g)
      if (kfs[g].empty()) {
        set_error("graph id %d has no keyframe", g);
        return MSLAM_ERR_ARG;
      }
    P->G = G;
    P->kf_off.assign(N + 1, 0);
    for (int k = 0; k < N; ++k) P->kf_off[k + 1] = P->kf_off[k] + (int64_t)kf_hw[2 * k] * kf_hw[2 * k + 1];
    P->e_off.assign(E + 1, 0);
    for (int e = 0; e < E; ++e) {
      const int i = edges[2 * e], j = edges[2 * e + 1];
      if (i < 0 || j < 0 || i >= N || j >= N || i == j || P->graph_of_kf[i] != P->graph_of_kf[j] ||
          kf_hw[2 * i] != kf_hw[2 * j] || kf_hw[2 * i + 1] != kf_hw[2 * j + 1]) {
        set_error("edge %d = (%d, %d): out of range, self edge, different graphs or sizes", e, i, j);
        return MSLAM_ERR_ARG;
      }
      const int H = kf_hw[2 * j], W = kf_hw[2 * j + 1];
      P->e_off[e + 1] = P->e_off[e] + (int64_t)H * W;
      DevEdge d{};
      d.i = i;
      d.j = j;
      d.H = H;
      d.W = W;
      d.off_e = P->e_off[e];
      d.off_i = P->kf_off[i];
      d.off_j = P->kf_off[j];
      d.graph = P->graph_of_kf[i];
      d.tile_begin = (int32_t)P->tiles.size();
      for (int b = 0; b < H * W; b += P->lin_tile) {
        DevTile t{};
        t.edge = e;
        t.begin = b;
        t.end = std::min(H * W, b + P->lin_tile);
        P->tiles.push_back(t);
      }
      d.tile_end = (int32_t)P->tiles.size();
      d.mblock_begin = P->n_mblocks;
      const int bh = P->match_by * P->match_ppt;  // rows of a match block
      P->n_mblocks += ((W + P->match_bx - 1) / P->match_bx) * ((H + bh - 1) / bh);
      P->dedges.push_back(d);
    }
    P->order.assign(N, -1);
    for (int g = 0; g < G; ++g) build_graph(P.get(), g, kfs[g]);
    size_t off = 0;
    P->off_edges = off;
    off = align256(off + sizeof(DevEdge) * P->dedges.size());
    P->off_tiles = off;
    off = align256(off + sizeof(DevTile) * P->tiles.size());
    P->off_graphs = off;
    off = align256(off + sizeof(DevGraph) * P->graphs.size());
    P->off_ints = off;
    off = align256(off + sizeof(int32_t) * P->ints.size());
    P->blob_bytes = std::max<size_t>(off, 256);
    *out = P.release();
    return MSLAM_OK;
  } catch (const std::exception& ex) {
    set_error("plan_create: host tables: %s", ex.what());
    return MSLAM_ERR_RANGE;
  }
}

void mslam_plan_destroy(mslam_plan* plan) { delete plan; }

size_t mslam_plan_device_bytes(const mslam_plan* plan) { return plan ? plan->blob_bytes : 0; }

mslam_status mslam_plan_upload(mslam_plan* plan, void* dev, size_t bytes, void* stream) {
  if (!plan || !dev || bytes < plan->blob_bytes || (reinterpret_cast<uintptr_t>(dev) & 255)) {
    set_error("plan upload: NULL plan/buffer, buffer smaller than %zu bytes, or not 256-byte aligned",
              plan ? plan->blob_bytes : (size_t)0);
    return MSLAM_ERR_ARG;
  }
  std::vector<char> blob(plan->blob_bytes, 0);
  std::memcpy(blob.data() + plan->off_edges, plan->dedges.data(), sizeof(DevEdge) * plan->dedges.size());
  std::memcpy(blob.data() + plan->off_tiles, plan->tiles.data(), sizeof(DevTile) * plan->tiles.size());
  std::memcpy(blob.data() + plan->off_graphs, plan->graphs.data(), sizeof(DevGraph) * plan->graphs.size());
  std::memcpy(blob.data() + plan->off_ints, plan->ints.data(), sizeof(int32_t) * plan->ints.size());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  mslam_status st = cuda_check(cudaMemcpyAsync(dev, blob.data(), blob.size(), cudaMemcpyHostToDevice, s),
                               "plan upload");
  if (st != MSLAM_OK) return st;
  // the staging vector is freed on return: wait for the copy out of it
  st = cuda_check(cudaStreamSynchronize(s), "plan upload sync");
  if (st != MSLAM_OK) return st;
  plan->dev = dev;
  plan->dev_bytes = bytes;
  return MSLAM_OK;
}

int64_t mslam_plan_kf_pixels(const mslam_plan* plan) { return plan ? plan->kf_off.back() : 0; }
int64_t mslam_plan_edge_pixels(const mslam_plan* plan) { return plan ? plan->e_off.back() : 0; }
int32_t mslam_plan_num_graphs(const mslam_plan* plan) { return plan ? plan->G : 0; }

void mslam_plan_offsets(const mslam_plan* plan, int64_t* kf_off, int64_t* e_off) {
  if (!plan) return;
  if (kf_off) std::copy(plan->kf_off.begin(), plan->kf_off.end(), kf_off);
  if (e_off) std::copy(plan->e_off.begin(), plan->e_off.end(), e_off);
}

void mslam_plan_stats(const mslam_plan* plan, int32_t* order, int64_t* counts) {
  if (!plan) return;
  if (order) std::copy(plan->order.begin(), plan->order.end(), order);
  if (counts) {
    counts[0] = plan->n_blocks_total;
    counts[1] = plan->n_trips_total;
    counts[2] = (int64_t)plan->tiles.size();
    counts[3] = plan->n_mblocks;
  }
}

size_t mslam_workspace_bytes(const mslam_plan* plan, int32_t op) {
  if (!plan) return 0;
  switch (op) {
    case MSLAM_OP_TRACK:
      // tile partials, then one completed-tile counter per edge
      return lin_partials_bytes((int)plan->tiles.size()) + align256(sizeof(int32_t) * std::max(plan->E, 1));
    case MSLAM_OP_LINEARIZE:
      // tile partials, relative poses, the tile counter
      return lin_partials_bytes((int)plan->tiles.size()) + align256(sizeof(float) * 16 * std::max(plan->E, 1)) + 256;
    case MSLAM_OP_SOLVE:  // per-graph FP64 blocks and vectors, then one flag per graph
      return align256(sizeof(double) * std::max<int64_t>(plan->solve_ws_doubles, 1)) +
             align256(sizeof(int32_t) * std::max<size_t>(plan->graphs.size(), 1));
    case MSLAM_OP_PACK_F32:
      return pack_bytes((int)plan->tiles.size(), plan->lin_tile, MSLAM_F32);
    case MSLAM_OP_PACK_F16:
      return pack_bytes((int)plan->tiles.size(), plan->lin_tile, MSLAM_F16);
    case MSLAM_OP_STATS:
      return align256(sizeof(uint32_t) * (size_t)((plan->e_off.back() + 31) / 32 + 1));
    case MSLAM_OP_MATCH:
      // the reference ray image (one float4 per edge-pool pixel), then the
      // keyframe-count bitmap (every edge starting on its own 32-bit word)
      return align256(sizeof(float) * 4 * (size_t)std::max<int64_t>(plan->e_off.back(), 1)) +
             align256(sizeof(uint32_t) * (size_t)((plan->e_off.back() + 32 * (int64_t)plan->E + 63) / 32 + 1));
    case MSLAM_OP_BACKWARD:
      // the solve's workspace, b and tau (7 N doubles each), per-edge data
      // (32 floats per edge), then for the pose term the step's right-hand
      // side and the pose gradient (7 N doubles each) and Xi (7 E doubles),
      // then one flag per graph for the second solve
      return mslam_workspace_bytes(plan, MSLAM_OP_SOLVE) + align256(sizeof(double) * 14 * (size_t)plan->N) +
             align256(sizeof(float) * 32 * (size_t)std::max(plan->E, 1)) +
             align256(sizeof(double) * (14 * (size_t)plan->N + 7 * (size_t)std::max(plan->E, 1))) +
             align256(sizeof(int32_t) * std::max<size_t>(plan->graphs.size(), 1));  // flags of the second solve
    default:
      return 0;
  }
}

}  // extern "C"
