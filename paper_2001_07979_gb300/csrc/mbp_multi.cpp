// Host driver of the grouped decode (mbp_decode_multi, mbp_autotune_multi and
// the MBP_SCHED_GRAPH schedule): workspace layout, per-group set-up, the CUDA
// graph of the iteration loop (built once per batch shape, workspace and launch
// shape, then cached) and the autotuner of the launch shapes.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "mbp_multi.h"

namespace mbp {

int multi_class_dmax(int d) {
  static const int bounds[] = {4, 6, 8, 10, 12, 14, 16, 18, 20, 22, 24, 32, 64};
  for (int b : bounds)
    if (d <= b) return b;
  return kMaxRowDeg;
}

namespace {

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Layout {
  int G = 0, T = 0, n_cls = 0;
  int cls_dmax[kMaxClasses] = {};
  std::vector<int> cls_of, tile_base, n_tiles;
  std::vector<size_t> group_off;
  size_t groups_off = 0, ctl_off = 0, tile_group_off = 0, lists_off = 0, pre_off = 0, tables_end = 0, total = 0;
};

int make_layout(const mbp_group* g, int G, int msg_dtype, bool host_io, Layout* L) {
  L->G = G;
  L->cls_of.assign(G, 0);
  L->tile_base.assign(G, 0);
  L->n_tiles.assign(G, 0);
  L->group_off.assign(G, 0);
  int64_t T = 0;
  for (int i = 0; i < G; ++i) {
    const int d = multi_class_dmax(g[i].codes->d.max_row_deg);
    int k = 0;
    while (k < L->n_cls && L->cls_dmax[k] != d) ++k;
    if (k == L->n_cls) {
      if (L->n_cls == kMaxClasses)
        return set_error(MBP_EUNSUPPORTED, "a batch may hold codes of at most %d check-degree classes", kMaxClasses);
      L->cls_dmax[L->n_cls++] = d;
    }
    L->cls_of[i] = k;
    L->tile_base[i] = int(T);
    L->n_tiles[i] = (g[i].F + kLanes - 1) / kLanes;
    T += L->n_tiles[i];
  }
  if (T > 65535) return set_error(MBP_EUNSUPPORTED, "a batch may hold at most %d frames", 65535 * kLanes);
  L->T = int(T);
  size_t o = 0;
  L->groups_off = o;
  o += align256(sizeof(MultiGroup) * size_t(G));
  L->ctl_off = o;
  o += align256(sizeof(MultiCtl));
  L->tile_group_off = o;
  o += align256(sizeof(int32_t) * size_t(T));
  L->tables_end = o;
  L->lists_off = o;
  o += align256(sizeof(int32_t) * size_t(L->n_cls + 1) * size_t(T));
  L->pre_off = o;
  o += align256(sizeof(int64_t) * size_t(2 * L->n_cls + 1) * size_t(T + 1));
  for (int i = 0; i < G; ++i) {
    L->group_off[i] = o;
    o += align256(workspace_bytes(g[i].codes->d, g[i].F, msg_dtype, host_io));
  }
  L->total = o;
  return MBP_OK;
}

MultiTables tables_at(const Layout& L, void* ws) {
  char* b = static_cast<char*>(ws);
  MultiTables tb;
  tb.groups = reinterpret_cast<MultiGroup*>(b + L.groups_off);
  tb.ctl = reinterpret_cast<MultiCtl*>(b + L.ctl_off);
  tb.tile_group = reinterpret_cast<int32_t*>(b + L.tile_group_off);
  tb.lists = reinterpret_cast<int32_t*>(b + L.lists_off);
  tb.pre = reinterpret_cast<int64_t*>(b + L.pre_off);
  return tb;
}

MultiShape shape_of(const Layout& L) {
  MultiShape sh;
  sh.G = L.G;
  sh.T = L.T;
  sh.n_cls = L.n_cls;
  for (int k = 0; k < kMaxClasses; ++k) sh.cls_dmax[k] = L.cls_dmax[k];
  return sh;
}

constexpr MultiTuning kDefaultTuning{1, 8, 1, 8, 8};

bool same_tuning(const MultiTuning& a, const MultiTuning& b) {
  return a.grid == b.grid && a.cn_warps == b.cn_warps && a.cn_waves == b.cn_waves && a.vn_warps == b.vn_warps &&
         a.syn_warps == b.syn_warps;
}

constexpr double kToInternal = 1.4426950408889634074;  // the FP32 decoder's internal unit: LLR x log2(e)

// Host copies of every group's code and state, for the grid kernels' launch parameters.
struct Groups {
  std::vector<DevCode> code;
  std::vector<DevState> st;
  double l_max;  // internal unit
};

// ---- kernel launches of one batch, by message type
struct Kernels {
  cudaError_t (*group_step)(const DevCode&, const DevState&, int, double, cudaStream_t, const StreamFork*);
  cudaError_t (*build_lists)(const MultiTables&, const MultiShape&, int, int, unsigned long long, const GroupConds&,
                             cudaStream_t);
  cudaError_t (*check)(const MultiTables&, const MultiShape&, int, const MultiTuning&, int, cudaStream_t);
  cudaError_t (*variable)(const MultiTables&, const MultiShape&, const MultiTuning&, int, cudaStream_t);
  cudaError_t (*syndrome)(const MultiTables&, const MultiShape&, int, const MultiTuning&, int, cudaStream_t);
};

template <typename S>
Kernels kernels_for() {
  return Kernels{&stream_group_step<float, S>, &MultiLaunch<S>::build_lists, &MultiLaunch<S>::check,
                 &MultiLaunch<S>::variable, &MultiLaunch<S>::syndrome};
}

Kernels kernels_of(int msg_dtype) {
  switch (msg_dtype) {
    case MBP_MSG_F16: return kernels_for<__half>();
    case MBP_MSG_BF16: return kernels_for<__nv_bfloat16>();
    default: return kernels_for<float>();
  }
}

const GroupConds kNoConds{0, {}};

// The test before iteration 1 and the retirement at t = 0: persistent kernels build the lists of every tile
// and run the class syndrome kernels over them; grid kernels run each group's stopping test.
cudaError_t issue_prologue(const Kernels& k, const MultiTables& tb, const MultiShape& sh, const MultiTuning& tu,
                           int sms, const Groups& gs, int in_graph, unsigned long long h, const GroupConds& gc,
                           cudaStream_t s) {
  cudaError_t e;
  if (tu.grid) {
    for (size_t g = 0; g < gs.code.size(); ++g) {
      if (gs.st[g].F == 0) continue;
      if ((e = k.group_step(gs.code[g], gs.st[g], kStopTestOnly, gs.l_max, s, nullptr)) != cudaSuccess) return e;
    }
    return k.build_lists(tb, sh, 2, in_graph, h, gc, s);
  }
  if ((e = k.build_lists(tb, sh, 0, 0, 0, kNoConds, s)) != cudaSuccess) return e;
  for (int c = 0; c < sh.n_cls; ++c)
    if ((e = k.syndrome(tb, sh, c, tu, sms, s)) != cudaSuccess) return e;
  return k.build_lists(tb, sh, 1, in_graph, h, gc, s);
}

// One iteration's decoding work: eq. (6) per class, eq. (2), the stopping test per class (persistent kernels);
// or every group's streaming-schedule kernels (grid kernels; iter = 1, 2 or 0 for a later iteration, fixed at
// capture: iteration 1 may leave its messages in row form, which iteration 2 reads).
cudaError_t issue_work(const Kernels& k, const MultiTables& tb, const MultiShape& sh, const MultiTuning& tu,
                       int sms, const Groups& gs, int iter, cudaStream_t s) {
  cudaError_t e;
  if (tu.grid) {
    for (size_t g = 0; g < gs.code.size(); ++g) {
      if (gs.st[g].F == 0) continue;
      if ((e = k.group_step(gs.code[g], gs.st[g], iter, gs.l_max, s, nullptr)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  prof_begin(MBP_KERNEL_CHECK, s);
  for (int c = 0; c < sh.n_cls; ++c)
    if ((e = k.check(tb, sh, c, tu, sms, s)) != cudaSuccess) return e;
  prof_end(MBP_KERNEL_CHECK, s, sh.n_cls);
  prof_begin(MBP_KERNEL_VARIABLE, s);
  if ((e = k.variable(tb, sh, tu, sms, s)) != cudaSuccess) return e;
  prof_end(MBP_KERNEL_VARIABLE, s, 1);
  prof_begin(MBP_KERNEL_SYNDROME, s);
  for (int c = 0; c < sh.n_cls; ++c)
    if ((e = k.syndrome(tb, sh, c, tu, sms, s)) != cudaSuccess) return e;
  prof_end(MBP_KERNEL_SYNDROME, s, sh.n_cls);
  return cudaSuccess;
}

// Retirement after an iteration; the grid kernels need no lists (retire mode 2).
cudaError_t issue_retire(const Kernels& k, const MultiTables& tb, const MultiShape& sh, const MultiTuning& tu,
                         int in_graph, unsigned long long h, const GroupConds& gc, cudaStream_t s) {
  prof_begin(MBP_KERNEL_RETIRE, s);
  const cudaError_t e = k.build_lists(tb, sh, tu.grid ? 2 : 1, in_graph, h, gc, s);
  prof_end(MBP_KERNEL_RETIRE, s, 1);
  return e;
}

// Grid kernels: one IF node per group with frames (parallel branches, each running its group's step while the
// group has unfinished tiles), all depending on `deps`; returns the IF nodes.
int add_group_branches(const Kernels& k, const Groups& gs, const GroupConds& gc, int iter, cudaGraph_t graph,
                       const std::vector<cudaGraphNode_t>& deps, cudaStream_t cs, const StreamFork* fork,
                       std::vector<cudaGraphNode_t>* nodes) {
  cudaError_t e;
  for (size_t g = 0; g < gs.code.size(); ++g) {
    if (gs.st[g].F == 0) continue;
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = gc.h[g];
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, graph, deps.data(), nullptr, deps.size(), &p)) != cudaSuccess)
      return cuda_error(e, "cudaGraphAddNode (IF)");
    cudaGraph_t sub = p.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cs, sub, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      return cuda_error(e, "begin capture (group step)");
    const cudaError_t ke = k.group_step(gs.code[g], gs.st[g], iter, gs.l_max, cs, fork);
    cudaGraph_t out = sub;
    const cudaError_t ee = cudaStreamEndCapture(cs, &out);
    if (ke != cudaSuccess) return cuda_error(ke, "group step during capture");
    if (ee != cudaSuccess) return cuda_error(ee, "end capture (group step)");
    nodes->push_back(node);
  }
  return MBP_OK;
}

// Capture `issue` into `graph` after `deps`; *leaf gets the captured work's last nodes.
template <typename F>
int capture_after(cudaGraph_t graph, const std::vector<cudaGraphNode_t>& deps, cudaStream_t cs, F issue,
                  std::vector<cudaGraphNode_t>* leaf, const char* what) {
  cudaError_t e;
  if ((e = cudaStreamBeginCaptureToGraph(cs, graph, deps.data(), nullptr, deps.size(),
                                         cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cuda_error(e, what);
  const cudaError_t ie = issue(cs);
  cudaStreamCaptureStatus status;
  const cudaGraphNode_t* d = nullptr;
  size_t nd = 0;
  const cudaError_t qe = cudaStreamGetCaptureInfo(cs, &status, nullptr, nullptr, &d, nullptr, &nd);
  if (leaf) leaf->assign(d, d + (qe == cudaSuccess ? nd : 0));
  cudaGraph_t out = graph;
  const cudaError_t ee = cudaStreamEndCapture(cs, &out);
  if (ie != cudaSuccess) return cuda_error(ie, what);
  if (qe != cudaSuccess) return cuda_error(qe, "cudaStreamGetCaptureInfo");
  if (ee != cudaSuccess) return cuda_error(ee, what);
  return MBP_OK;
}

// The whole loop as one graph. Persistent kernels: the prologue, then a WHILE node whose body is one
// iteration. Grid kernels: the prologue, iterations 1 and 2, then WHILE{iteration}, where each iteration is
// one IF node per group (its step runs only while the group has unfinished tiles; the groups run as parallel
// branches) followed by the retire kernel, which sets the WHILE and IF conditions for the next iteration.
int build_graph(const Kernels& k, const MultiTables& tb, const MultiShape& sh, const MultiTuning& tu, int sms,
                const Groups& gs, cudaGraphExec_t* out) {
  cudaError_t e;
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  int rc = MBP_OK;
  GroupConds ga{0, {}}, g2{0, {}}, gb{0, {}};  // IF conditions of iterations 1, 2 and of the loop body
  std::vector<cudaGraphNode_t> leaf, branches;
  StreamFork fork{};  // the variable-node classes of a group step as parallel branches
#define GK(call, what)                 \
  if ((e = (call)) != cudaSuccess) {   \
    rc = cuda_error(e, what);          \
    goto done;                         \
  }
#define GR(call)           \
  if ((rc = (call))) goto done;
  {
    GK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
    GK(cudaStreamCreateWithFlags(&fork.aux[0], cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
    GK(cudaStreamCreateWithFlags(&fork.aux[1], cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
    GK(cudaEventCreateWithFlags(&fork.fork, cudaEventDisableTiming), "cudaEventCreateWithFlags");
    GK(cudaEventCreateWithFlags(&fork.join[0], cudaEventDisableTiming), "cudaEventCreateWithFlags");
    GK(cudaEventCreateWithFlags(&fork.join[1], cudaEventDisableTiming), "cudaEventCreateWithFlags");
    GK(cudaGraphCreate(&g, 0), "cudaGraphCreate");
    cudaGraphConditionalHandle h;
    GK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault), "cudaGraphConditionalHandleCreate");
    if (tu.grid) {
      ga.n = g2.n = gb.n = int(gs.code.size());
      for (size_t q = 0; q < gs.code.size(); ++q) {
        ga.h[q] = g2.h[q] = gb.h[q] = ~0ull;
        if (gs.st[q].F == 0) continue;
        cudaGraphConditionalHandle ha, h2, hb;
        GK(cudaGraphConditionalHandleCreate(&ha, g, 1, cudaGraphCondAssignDefault), "conditional handle (IF)");
        GK(cudaGraphConditionalHandleCreate(&h2, g, 1, cudaGraphCondAssignDefault), "conditional handle (IF)");
        GK(cudaGraphConditionalHandleCreate(&hb, g, 1, cudaGraphCondAssignDefault), "conditional handle (IF)");
        ga.h[q] = ha;
        g2.h[q] = h2;
        gb.h[q] = hb;
      }
    }
    GR(capture_after(g, {}, cs, [&](cudaStream_t st) { return issue_prologue(k, tb, sh, tu, sms, gs, 1, h, ga, st); },
                     &leaf, "capture (prologue)"));
    if (tu.grid) {  // iterations 1 and 2
      branches.clear();
      GR(add_group_branches(k, gs, ga, 1, g, leaf, cs, &fork, &branches));
      GR(capture_after(g, branches, cs, [&](cudaStream_t st) { return issue_retire(k, tb, sh, tu, 1, h, g2, st); },
                       &leaf, "capture (retire)"));
      branches.clear();
      GR(add_group_branches(k, gs, g2, 2, g, leaf, cs, &fork, &branches));
      GR(capture_after(g, branches, cs, [&](cudaStream_t st) { return issue_retire(k, tb, sh, tu, 1, h, gb, st); },
                       &leaf, "capture (retire)"));
    }
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t cnode;
    GK(cudaGraphAddNode(&cnode, g, leaf.data(), nullptr, leaf.size(), &p), "cudaGraphAddNode (WHILE)");
    cudaGraph_t body = p.conditional.phGraph_out[0];
    if (tu.grid) {
      branches.clear();
      GR(add_group_branches(k, gs, gb, 0, body, {}, cs, &fork, &branches));
      GR(capture_after(body, branches, cs, [&](cudaStream_t st) { return issue_retire(k, tb, sh, tu, 1, h, gb, st); },
                       nullptr, "capture (loop body)"));
    } else {
      GR(capture_after(body, {}, cs,
                       [&](cudaStream_t st) {
                         cudaError_t we = issue_work(k, tb, sh, tu, sms, gs, 0, st);
                         return we != cudaSuccess ? we : issue_retire(k, tb, sh, tu, 1, h, kNoConds, st);
                       },
                       nullptr, "capture (loop body)"));
    }
    GK(cudaGraphInstantiate(out, g, 0), "cudaGraphInstantiate");
  }
done:
#undef GR
#undef GK
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  for (cudaStream_t a : fork.aux)
    if (a) cudaStreamDestroy(a);
  for (cudaEvent_t ev : {fork.fork, fork.join[0], fork.join[1]})
    if (ev) cudaEventDestroy(ev);
  return rc;
}

// ---- caches: instantiated graphs, and the tuned launch shape of each batch signature
struct GraphEntry {
  int device;
  const void* ws;
  int msg_dtype;
  MultiShape sh;
  MultiTuning tu;
  double l_max;
  std::vector<const DevCode*> codes;  // the grid kernels take each group's code and state as parameters
  std::vector<int> F;
  std::vector<DevState> st;  // every group's state as captured (workspace carving, LLR or BSC inputs)
  cudaGraphExec_t exec;
  uint64_t used;
};

struct TuneEntry {
  int device, msg_dtype;
  std::vector<const void*> codes;
  std::vector<int> F;
  MultiTuning tu;
};

std::mutex g_mu;
std::vector<GraphEntry> g_graphs;
std::vector<TuneEntry> g_tuned;
uint64_t g_clock = 0;
constexpr size_t kMaxGraphs = 16;

static_assert(std::is_trivially_copyable<DevState>::value, "DevState is compared bytewise");

bool same_states(const std::vector<DevState>& a, const std::vector<DevState>& b) {
  return a.size() == b.size() && (a.empty() || std::memcmp(a.data(), b.data(), a.size() * sizeof(DevState)) == 0);
}

bool same_shape(const MultiShape& a, const MultiShape& b) {
  if (a.G != b.G || a.T != b.T || a.n_cls != b.n_cls) return false;
  for (int k = 0; k < a.n_cls; ++k)
    if (a.cls_dmax[k] != b.cls_dmax[k]) return false;
  return true;
}

int graph_for(const Kernels& k, int device, void* ws, int msg_dtype, const MultiTables& tb, const MultiShape& sh,
              const MultiTuning& tu, int sms, const Groups& gs, const std::vector<const DevCode*>& codes,
              cudaGraphExec_t* out) {
  std::vector<int> F;
  for (const auto& st : gs.st) F.push_back(st.F);
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto& ge : g_graphs)
    if (ge.device == device && ge.ws == ws && ge.msg_dtype == msg_dtype && same_shape(ge.sh, sh) &&
        same_tuning(ge.tu, tu) && ge.l_max == gs.l_max && ge.codes == codes && ge.F == F &&
        same_states(ge.st, gs.st)) {
      ge.used = ++g_clock;
      *out = ge.exec;
      return MBP_OK;
    }
  cudaGraphExec_t exec = nullptr;
  const int rc = build_graph(k, tb, sh, tu, sms, gs, &exec);
  if (rc) return rc;
  if (g_graphs.size() >= kMaxGraphs) {
    auto lru = std::min_element(g_graphs.begin(), g_graphs.end(),
                                [](const GraphEntry& a, const GraphEntry& b) { return a.used < b.used; });
    cudaGraphExecDestroy(lru->exec);
    g_graphs.erase(lru);
  }
  g_graphs.push_back(GraphEntry{device, ws, msg_dtype, sh, tu, gs.l_max, codes, F, gs.st, exec, ++g_clock});
  *out = exec;
  return MBP_OK;
}

bool tuned_for(int device, int msg_dtype, const mbp_group* g, int G, MultiTuning* tu) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (const auto& te : g_tuned) {
    if (te.device != device || te.msg_dtype != msg_dtype || int(te.codes.size()) != G) continue;
    bool same = true;
    for (int i = 0; i < G && same; ++i) same = te.codes[i] == g[i].codes && te.F[i] == g[i].F;
    if (same) {
      *tu = te.tu;
      return true;
    }
  }
  return false;
}

void remember_tuning(int device, int msg_dtype, const mbp_group* g, int G, const MultiTuning& tu) {
  std::lock_guard<std::mutex> lock(g_mu);
  TuneEntry te{device, msg_dtype, {}, {}, tu};
  for (int i = 0; i < G; ++i) {
    te.codes.push_back(g[i].codes);
    te.F.push_back(g[i].F);
  }
  for (auto& old : g_tuned)
    if (old.device == device && old.msg_dtype == msg_dtype && old.codes == te.codes && old.F == te.F) {
      old.tu = tu;
      return;
    }
  if (g_tuned.size() >= 64) g_tuned.erase(g_tuned.begin());
  g_tuned.push_back(std::move(te));
}

int sm_count(int* device, int* sms) {
  cudaError_t e;
  if ((e = cudaGetDevice(device)) != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, *device)) != cudaSuccess)
    return cuda_error(e, "cudaDeviceGetAttribute");
  return MBP_OK;
}

int run_multi(const mbp_group* g, int G, int max_iter, const mbp_opts* o, bool host_io, const MultiTuning* force,
              cudaStream_t s) {
  Layout L;
  int rc = make_layout(g, G, o->msg_dtype, host_io, &L);
  if (rc) return rc;
  if (L.total > o->workspace_bytes)
    return set_error(MBP_EINVAL, "workspace of %zu bytes is smaller than the %zu this batch needs",
                     o->workspace_bytes, L.total);
  if (L.T == 0) return MBP_OK;
  int device = 0, sms = 0;
  if ((rc = sm_count(&device, &sms))) return rc;
  MultiTuning tu = kDefaultTuning;
  if (force) tu = *force;
  else tuned_for(device, o->msg_dtype, g, G, &tu);
  const MultiTables tb = tables_at(L, o->workspace);
  const MultiShape sh = shape_of(L);
  const Kernels k = kernels_of(o->msg_dtype);
  // host copies of the tables: groups, control block, tile -> group
  std::vector<unsigned char> host(L.tables_end, 0);
  MultiGroup* hg = reinterpret_cast<MultiGroup*>(host.data() + L.groups_off);
  std::vector<DevState> st(G);
  Groups gs;
  gs.l_max = o->l_max * kToInternal;
  std::vector<const DevCode*> code_ids;
  for (int i = 0; i < G; ++i) {
    carve_workspace(g[i].codes->d, g[i].F, o->msg_dtype, host_io, static_cast<char*>(o->workspace) + L.group_off[i],
                    &st[i]);
    if (g[i].llr) st[i].yt = nullptr;  // L_P from the LLR array, not from sign words
    gs.code.push_back(g[i].codes->d);
    gs.st.push_back(st[i]);
    code_ids.push_back(&g[i].codes->d);
    hg[i].c = g[i].codes->d;
    hg[i].st = st[i];
    hg[i].tile_base = L.tile_base[i];
    hg[i].cls = L.cls_of[i];
    hg[i].iters = g[i].iters;
    hg[i].success = g[i].success;
    hg[i].synd_ok = g[i].synd_ok;
  }
  MultiCtl* hc = reinterpret_cast<MultiCtl*>(host.data() + L.ctl_off);
  hc->t = 0;
  hc->max_iter = max_iter;
  hc->early_exit = o->early_exit;
  hc->cond = 0;
  hc->l_max = float(o->l_max * kToInternal);
  int32_t* htg = reinterpret_cast<int32_t*>(host.data() + L.tile_group_off);
  for (int i = 0; i < G; ++i)
    for (int t = 0; t < L.n_tiles[i]; ++t) htg[L.tile_base[i] + t] = i;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(o->workspace, host.data(), host.size(), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_error(e, "copy batch tables");
  // set-up of every group (channel LLRs, syndrome words, tile state)
  for (int i = 0; i < G; ++i) {
    if (g[i].F == 0) continue;
    DecodeArgs a{};
    a.llr = g[i].llr;
    a.y_bits = g[i].llr ? nullptr : g[i].y_bits;
    a.qber = g[i].qber;
    a.z_bits = g[i].z_bits;
    a.max_iter = max_iter;
    a.early_exit = o->early_exit;
    a.validate = o->validate;
    a.l_max = o->l_max;
    a.x_hat_bits = g[i].x_hat_bits;
    a.iters = g[i].iters;
    a.success = g[i].success;
    a.soft_out = g[i].soft_out;
    a.synd_ok = g[i].synd_ok;
    if ((rc = group_setup(g[i].codes->d, st[i], o->msg_dtype, a, s))) return rc;
  }
  if (prof_on()) {
    // host-driven loop: the same kernels, one launch each, with a read-back of the loop condition
    int32_t cond = 0;
    prof_begin(MBP_KERNEL_RETIRE, s);
    if ((e = issue_prologue(k, tb, sh, tu, sms, gs, 0, 0, kNoConds, s)) != cudaSuccess)
      return cuda_error(e, "grouped prologue");
    int pro = 2 + sh.n_cls;
    if (tu.grid) {
      pro = 1;
      for (const auto& q : gs.st) pro += q.F > 0;
    }
    prof_end(MBP_KERNEL_RETIRE, s, pro);
    for (int t = 1;; ++t) {
      if ((e = cudaMemcpyAsync(&cond, &tb.ctl->cond, sizeof cond, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_error(e, "read loop condition");
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
      if (!cond) break;
      if ((e = issue_work(k, tb, sh, tu, sms, gs, t <= 2 ? t : 0, s)) != cudaSuccess) return cuda_error(e, "grouped iteration");
      if ((e = issue_retire(k, tb, sh, tu, 0, 0, kNoConds, s)) != cudaSuccess) return cuda_error(e, "grouped retire");
    }
  } else {
    cudaGraphExec_t exec = nullptr;
    if ((rc = graph_for(k, device, o->workspace, o->msg_dtype, tb, sh, tu, sms, gs, code_ids, &exec))) return rc;
    if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
  }
  for (int i = 0; i < G; ++i) {
    if (g[i].F == 0) continue;
    DecodeArgs a{};
    a.x_hat_bits = g[i].x_hat_bits;
    a.iters = g[i].iters;
    a.soft_out = g[i].soft_out;
    if ((rc = group_output(g[i].codes->d, st[i], o->msg_dtype, a, s))) return rc;
  }
  return MBP_OK;
}

}  // namespace

int multi_check_opts(const mbp_opts* o) {
  if (o->rule != MBP_RULE_SUM_PRODUCT || o->update != MBP_UPDATE_FLOODING)
    return set_error(MBP_EUNSUPPORTED, "the grouped (graph) decode runs the flooding sum-product decoder");
  if (o->msg_dtype == MBP_MSG_F64)
    return set_error(MBP_EUNSUPPORTED, "the grouped (graph) decode stores FP32, FP16 or BF16 messages");
  if (o->accumulate == MBP_ACC_FIXED)
    return set_error(MBP_EUNSUPPORTED, "the grouped (graph) decode accumulates in floating point only");
  return MBP_OK;
}

int multi_workspace(const mbp_group* g, int G, const mbp_opts* o, bool host_io, size_t* bytes) {
  Layout L;
  const int rc = make_layout(g, G, o->msg_dtype, host_io, &L);
  if (rc) return rc;
  *bytes = L.total;
  return MBP_OK;
}

int multi_group_state(const mbp_group* g, int G, int index, const mbp_opts* o, bool host_io, DevState* st) {
  Layout L;
  const int rc = make_layout(g, G, o->msg_dtype, host_io, &L);
  if (rc) return rc;
  carve_workspace(g[index].codes->d, g[index].F, o->msg_dtype, host_io,
                  static_cast<char*>(o->workspace) + L.group_off[index], st);
  return MBP_OK;
}

int multi_decode(const mbp_group* g, int G, int max_iter, const mbp_opts* o, bool host_io, cudaStream_t s) {
  return run_multi(g, G, max_iter, o, host_io, nullptr, s);
}

// Coordinate search over the launch shapes: the check-node kernels' block size
// and grid, then the variable-node kernel's block size. Each candidate decodes
// the batch once to build (and warm) its graph and is then timed over one more
// decode with CUDA events on the stream.
int multi_autotune(const mbp_group* g, int G, int max_iter, const mbp_opts* o, mbp_tuning* best_out,
                   cudaStream_t s) {
  int device = 0, sms = 0;
  int rc = sm_count(&device, &sms);
  if (rc) return rc;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return cuda_error(e, "cudaEventCreate");
  if ((e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_error(e, "cudaEventCreate");
  }
  const bool was_prof = prof_on();
  if (was_prof) prof_enable(false);
  auto time_one = [&](const MultiTuning& tu, float* ms) -> int {
    int r = run_multi(g, G, max_iter, o, false, &tu, s);
    if (r) return r;
    if ((e = cudaEventRecord(a, s)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    if ((r = run_multi(g, G, max_iter, o, false, &tu, s))) return r;
    if ((e = cudaEventRecord(b, s)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) return cuda_error(e, "cudaEventSynchronize");
    if ((e = cudaEventElapsedTime(ms, a, b)) != cudaSuccess) return cuda_error(e, "cudaEventElapsedTime");
    return MBP_OK;
  };
  MultiTuning best = kDefaultTuning;
  float best_ms = 0.f;
  rc = time_one(best, &best_ms);
  if (!rc) {  // grid kernels (the default) against the persistent list kernels
    MultiTuning tu = best;
    tu.grid = 0;
    float ms = 0.f;
    rc = time_one(tu, &ms);
    if (!rc && ms < best_ms) {
      best = tu;
      best_ms = ms;
    }
  }
  static const int warps[] = {2, 4, 8};
  for (int w : warps)
    for (int waves = 1; waves <= 2 && !rc && !best.grid; ++waves) {
      MultiTuning tu = best;
      tu.cn_warps = w;
      tu.cn_waves = waves;
      if (same_tuning(tu, best)) continue;
      float ms = 0.f;
      rc = time_one(tu, &ms);
      if (!rc && ms < best_ms) {
        best = tu;
        best_ms = ms;
      }
    }
  for (int w : warps) {
    if (rc || best.grid) break;
    MultiTuning tu = best;
    tu.vn_warps = w;
    tu.syn_warps = w;
    if (same_tuning(tu, best)) continue;
    float ms = 0.f;
    rc = time_one(tu, &ms);
    if (!rc && ms < best_ms) {
      best = tu;
      best_ms = ms;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (was_prof) prof_enable(true);
  if (rc) return rc;
  remember_tuning(device, o->msg_dtype, g, G, best);
  if (best_out) {
    best_out->grid_kernels = best.grid;
    best_out->cn_warps = best.cn_warps;
    best_out->cn_waves = best.cn_waves;
    best_out->vn_warps = best.vn_warps;
    best_out->syn_warps = best.syn_warps;
    best_out->ms = best_ms;
  }
  // leave the outputs of a decode with the chosen shape
  return run_multi(g, G, max_iter, o, false, &best, s);
}

int multi_set_tuning(const mbp_group* g, int G, const mbp_opts* o, const mbp_tuning* t) {
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  MultiTuning tu{t->grid_kernels ? 1 : 0, t->cn_warps, t->cn_waves, t->vn_warps, t->syn_warps};
  remember_tuning(device, o->msg_dtype, g, G, tu);
  return MBP_OK;
}

void multi_release() {
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto& ge : g_graphs) cudaGraphExecDestroy(ge.exec);
  g_graphs.clear();
  g_tuned.clear();
}

void multi_forget(const mbp_codes* h) {
  std::lock_guard<std::mutex> lock(g_mu);
  const DevCode* d = &h->d;
  for (size_t i = g_graphs.size(); i-- > 0;)
    if (std::find(g_graphs[i].codes.begin(), g_graphs[i].codes.end(), d) != g_graphs[i].codes.end()) {
      cudaGraphExecDestroy(g_graphs[i].exec);
      g_graphs.erase(g_graphs.begin() + i);
    }
  for (size_t i = g_tuned.size(); i-- > 0;)
    if (std::find(g_tuned[i].codes.begin(), g_tuned[i].codes.end(), static_cast<const void*>(h)) !=
        g_tuned[i].codes.end())
      g_tuned.erase(g_tuned.begin() + i);
}

}  // namespace mbp
