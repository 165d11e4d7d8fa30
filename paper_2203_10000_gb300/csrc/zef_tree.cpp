// zef_tree.cpp -- exact far-field replacement of surface patches by caps.
//
// A compartment's triangles are split recursively (median of the triangle
// centroids along the longest axis of their box) into a binary tree of
// patches down to leaves of at most kCapLeaf triangles.  Every patch P other
// than the whole (closed) surface has a boundary: the directed edges u -> v
// of its triangles whose opposite v -> u belongs to no triangle of P; they
// form closed loops u0 -> u1 -> ... -> u(m-1) -> u0.  P's cap triangulates
// each loop with vertices of the loop only: the triangles (u_i, u_j, u_k),
// i < j < k, of the zigzag order u0, u(m-1), u1, u(m-2), u2, ...  Their
// interior edges cancel in pairs, so the cap has the same directed boundary
// as P and P together with the reversed cap is a closed surface.  All its
// vertices are vertices of P, so it lies in the box of P, and its winding
// number is 0 at every point outside that box: there the solid angle of P
// equals the solid angle of the cap exactly (Sec. 2.1.3: Omega of a closed
// surface is 4 pi times the winding number).  A point tile whose box misses
// the box of P sums P's cap instead of P's triangles.
//
// Both the leaves' triangles and the caps are stored as strip segments of
// the Entry format of the surface strips: the vertex entering the sliding
// window (weight +1 / -1 when the window (previous two vertices, this one)
// is a triangle in its own / the reversed orientation, 0 otherwise) and the
// triangle's doubled-area normal with kappa |n|.  A segment starts with a
// reset entry (weight 2: the window restarts at that vertex, the entry's own
// window (x0, x0, x0) is an identity factor) and is padded with identity
// windows to a multiple of four entries.  Leaves are covered by greedy
// strips that may turn either way: a turn costs one repeated vertex (window
// (p, q, p)), a new strip four (windows (y, z, z), (z, z, x0), (z, x0, x0),
// (x0, x0, x1)).  Every non-triangle window repeats a vertex, so its N is 0
// and its D >= 0: a positive real factor.
//
// Layout per compartment: the nodes in pre-order (a node's left child is the
// next node, and `skip` is the node after its subtree, so walks need no
// stack); the leaf segments in tree order, then the cap segments of all its
// nodes (the leaves' block alone is the whole surface); the triangle indices
// in leaf order (a leaf's triangles for box queries such as the inflation's).
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstring>
#include <unordered_set>
#include <vector>

#include "zef_internal.h"

namespace zef {

namespace {

inline uint64_t dkey(int32_t u, int32_t v) { return ((uint64_t)(uint32_t)u << 32) | (uint32_t)v; }

// One entry of a strip: the vertex and, when its window is a triangle, that
// triangle with its own orientation.
struct Item {
  int32_t v;
  bool tri;
  std::array<int32_t, 3> o;
};

// Writes strips into one segment.
struct SegWriter {
  const float *V;
  std::vector<Entry> *out;
  size_t begin = 0;
  int32_t last = -1;         // last vertex written
  int32_t w1 = -1, w2 = -1;  // the current window (for the orientation sign)
  int64_t tris = 0;

  Entry ent(int32_t v, float w) const {
    Entry e;
    e.v = make_float4(V[3 * (int64_t)v], V[3 * (int64_t)v + 1], V[3 * (int64_t)v + 2], w);
    e.n = make_float4(0.f, 0.f, 0.f, 0.f);
    return e;
  }
  void push(int32_t v, float w) {
    out->push_back(ent(v, w));
    w1 = w2;
    w2 = v;
    last = v;
  }
  void push_tri(int32_t c, const std::array<int32_t, 3> &o) {
    // +1 when the window (w1, w2, c) is a rotation of o, -1 when reversed
    int ia = 0;
    while (ia < 3 && o[(size_t)ia] != w1) ++ia;
    const float w = (ia < 3 && o[(size_t)((ia + 1) % 3)] == w2) ? 1.f : -1.f;
    Entry e = ent(c, w);
    double p[3][3];
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) p[k][d] = V[3 * (int64_t)o[(size_t)k] + d];
    double e1[3], e2[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = p[1][d] - p[0][d];
      e2[d] = p[2][d] - p[0][d];
    }
    const double nx = e1[1] * e2[2] - e1[2] * e2[1];
    const double ny = e1[2] * e2[0] - e1[0] * e2[2];
    const double nz = e1[0] * e2[1] - e1[1] * e2[0];
    e.n = make_float4((float)nx, (float)ny, (float)nz, (float)(kKappa * std::sqrt(nx * nx + ny * ny + nz * nz)));
    out->push_back(e);
    w1 = w2;
    w2 = c;
    last = c;
    ++tris;
  }
  // a strip: items[0] and items[1] open the window, the rest follow
  void strip(const std::vector<Item> &items) {
    if (last < 0) {
      begin = out->size();
      push(items[0].v, 2.f);  // reset
    } else {
      push(last, 0.f);
      push(items[0].v, 0.f);
      push(items[0].v, 0.f);
    }
    for (size_t k = 1; k < items.size(); ++k) {
      if (items[k].tri) push_tri(items[k].v, items[k].o);
      else push(items[k].v, 0.f);
    }
  }
  void finish() {
    if (last < 0) return;
    while ((out->size() - begin) % 4) push(last, 0.f);
    last = -1;
  }
};

// Greedy strips with turns over a small set of oriented triangles (a leaf).
void leaf_strips(const int32_t *T, const std::vector<int64_t> &tris, SegWriter &w) {
  const int n = (int)tris.size();
  auto f = [&](int t, int k) { return T[3 * tris[(size_t)t] + (k % 3)]; };
  // nb[t][k]: the triangle across edge (f(t,k), f(t,k+1)), -1 if outside
  std::vector<std::array<int, 3>> nb((size_t)n, {-1, -1, -1});
  std::vector<std::pair<uint64_t, int>> dir;  // directed edge -> its triangle
  for (int t = 0; t < n; ++t)
    for (int k = 0; k < 3; ++k) dir.push_back({dkey(f(t, k), f(t, k + 1)), t});
  std::sort(dir.begin(), dir.end());
  for (int t = 0; t < n; ++t)
    for (int k = 0; k < 3; ++k) {
      const uint64_t rev = dkey(f(t, k + 1), f(t, k));
      auto it = std::lower_bound(dir.begin(), dir.end(), std::make_pair(rev, INT_MIN));
      if (it != dir.end() && it->first == rev) nb[(size_t)t][(size_t)k] = it->second;
    }
  auto across = [&](int t, int32_t a, int32_t b) {  // neighbour of t across edge {a, b}
    for (int k = 0; k < 3; ++k)
      if ((f(t, k) == a && f(t, k + 1) == b) || (f(t, k) == b && f(t, k + 1) == a)) return nb[(size_t)t][(size_t)k];
    return -1;
  };
  auto third = [&](int t, int32_t a, int32_t b) {
    for (int k = 0; k < 3; ++k)
      if (f(t, k) != a && f(t, k) != b) return f(t, k);
    return (int32_t)-1;
  };
  auto orient = [&](int t) { return std::array<int32_t, 3>{f(t, 0), f(t, 1), f(t, 2)}; };
  // walk from triangle t0 entered with window (f(t0,r), f(t0,r+1)): the
  // items and the triangles taken (`used` is not modified)
  auto walk = [&](int t0, int r, const std::vector<uint8_t> &used, std::vector<Item> &items,
                  std::vector<int> &taken) {
    items.clear();
    taken.clear();
    std::vector<uint8_t> u(used);
    int32_t p = f(t0, r), q = f(t0, r + 1);
    items.push_back({p, false, {}});
    items.push_back({q, false, {}});
    int t = t0;
    for (;;) {
      u[(size_t)t] = 1;
      taken.push_back(t);
      const int32_t x = third(t, p, q);
      const int s = across(t, q, x);
      if (s >= 0 && !u[(size_t)s]) {  // straight on: exit edge (q, x)
        items.push_back({x, true, orient(t)});
        p = q;
        q = x;
        t = s;
        continue;
      }
      const int s2 = across(t, p, x);
      if (s2 >= 0 && !u[(size_t)s2]) {  // turn: (p, q, p) then (q, p, x); exit edge (p, x)
        items.push_back({p, false, {}});
        items.push_back({x, true, orient(t)});
        q = x;
        t = s2;
        continue;
      }
      items.push_back({x, true, orient(t)});
      break;
    }
  };
  std::vector<uint8_t> used((size_t)n, 0);
  std::vector<Item> items, best_items;
  std::vector<int> taken, best_taken;
  for (;;) {
    // start at the unused triangle with the fewest unused neighbours
    int t0 = -1, deg0 = 4;
    for (int t = 0; t < n; ++t) {
      if (used[(size_t)t]) continue;
      int d = 0;
      for (int k = 0; k < 3; ++k) {
        const int s = nb[(size_t)t][(size_t)k];
        d += s >= 0 && !used[(size_t)s];
      }
      if (d < deg0) {
        deg0 = d;
        t0 = t;
      }
    }
    if (t0 < 0) break;
    best_items.clear();
    best_taken.clear();
    for (int r = 0; r < 3; ++r) {
      walk(t0, r, used, items, taken);
      // most triangles, then fewest entries
      if (taken.size() > best_taken.size() ||
          (taken.size() == best_taken.size() && items.size() < best_items.size())) {
        best_items = items;
        best_taken = taken;
      }
    }
    for (int t : best_taken) used[(size_t)t] = 1;
    w.strip(best_items);
  }
  w.finish();
}

// Zigzag triangulations of the loops of a set of directed boundary edges.
void cap_strips(const std::vector<std::pair<int32_t, int32_t>> &boundary, SegWriter &w) {
  std::vector<std::pair<int32_t, int32_t>> edges(boundary);
  std::sort(edges.begin(), edges.end());
  std::vector<uint8_t> used(edges.size(), 0);
  for (size_t e0 = 0; e0 < edges.size(); ++e0) {
    if (used[e0]) continue;
    // a closed walk along unused edges (each vertex of a closed surface's
    // patch boundary has as many boundary edges leaving as entering it)
    std::vector<int32_t> loop;
    size_t e = e0;
    for (;;) {
      used[e] = 1;
      loop.push_back(edges[e].first);
      const int32_t v = edges[e].second;
      if (v == edges[e0].first) break;
      auto it = std::lower_bound(edges.begin(), edges.end(), std::make_pair(v, (int32_t)INT32_MIN));
      size_t nx = edges.size();
      for (; it != edges.end() && it->first == v; ++it)
        if (!used[(size_t)(it - edges.begin())]) {
          nx = (size_t)(it - edges.begin());
          break;
        }
      if (nx == edges.size()) break;
      e = nx;
    }
    const int m = (int)loop.size();
    if (m < 3) continue;
    std::vector<int> pos;  // zigzag order of loop positions
    for (int lo = 0, hi = m - 1, k = 0; lo <= hi; ++k) pos.push_back(k % 2 == 0 ? lo++ : hi--);
    std::vector<Item> items;
    for (int k = 0; k < m; ++k) {
      Item it{loop[(size_t)pos[(size_t)k]], k >= 2, {}};
      if (k >= 2) {
        int p3[3] = {pos[(size_t)k - 2], pos[(size_t)k - 1], pos[(size_t)k]};
        std::sort(p3, p3 + 3);
        it.o = {loop[(size_t)p3[0]], loop[(size_t)p3[1]], loop[(size_t)p3[2]]};
      }
      items.push_back(it);
    }
    w.strip(items);
  }
  w.finish();
}

struct Builder {
  const float *V;
  const int32_t *T;
  std::vector<CapNode> *nodes;
  std::vector<Entry> leaf_seg;  // leaf segments, tree order
  std::vector<Entry> cap_seg;   // cap segments
  std::vector<int64_t> idx;
  std::vector<double> cen;      // 3 per triangle

  // acc := directed boundary of acc + more: a directed edge whose opposite is
  // present cancels with it; the result is sorted (deterministic cap order)
  static void cancel_into(std::vector<std::pair<int32_t, int32_t>> &acc,
                          const std::vector<std::pair<int32_t, int32_t>> &more) {
    std::unordered_set<uint64_t> s;
    s.reserve((acc.size() + more.size()) * 2 + 16);
    auto add = [&](const std::pair<int32_t, int32_t> &e) {
      if (s.erase(dkey(e.second, e.first)) == 0) s.insert(dkey(e.first, e.second));
    };
    for (auto &e : acc) add(e);
    for (auto &e : more) add(e);
    std::vector<uint64_t> keys(s.begin(), s.end());
    std::sort(keys.begin(), keys.end());
    acc.clear();
    for (uint64_t k : keys) acc.push_back({(int32_t)(uint32_t)(k >> 32), (int32_t)(uint32_t)(k & 0xffffffffu)});
  }

  int32_t build(int64_t b, int64_t e, std::vector<std::pair<int32_t, int32_t>> &boundary) {
    const int32_t me = (int32_t)nodes->size();
    nodes->push_back(CapNode{});
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t k = b; k < e; ++k)
      for (int q = 0; q < 3; ++q) {
        const float *p = V + 3 * (int64_t)T[3 * idx[k] + q];
        for (int d = 0; d < 3; ++d) {
          lo[d] = std::min(lo[d], p[d]);
          hi[d] = std::max(hi[d], p[d]);
        }
      }
    CapNode node{};
    node.left = node.right = -1;
    if (e - b <= kCapLeaf) {
      std::vector<std::pair<int32_t, int32_t>> edges;
      for (int64_t k = b; k < e; ++k) {
        const int32_t *t = T + 3 * idx[k];
        edges.push_back({t[0], t[1]});
        edges.push_back({t[1], t[2]});
        edges.push_back({t[2], t[0]});
      }
      boundary.clear();
      cancel_into(boundary, edges);
      std::vector<int64_t> mine(idx.begin() + b, idx.begin() + e);
      SegWriter sw{V, &leaf_seg};
      node.tri_begin = (int32_t)b;
      node.leaf_begin = (int32_t)leaf_seg.size();
      leaf_strips(T, mine, sw);
      node.leaf_cnt = (int32_t)leaf_seg.size() - node.leaf_begin;
      node.leaf_tris = (int32_t)sw.tris;
    } else {
      // median split of the centroids along the longest axis of their box
      double cl[3] = {INFINITY, INFINITY, INFINITY}, ch[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int64_t k = b; k < e; ++k)
        for (int d = 0; d < 3; ++d) {
          cl[d] = std::min(cl[d], cen[3 * idx[k] + d]);
          ch[d] = std::max(ch[d], cen[3 * idx[k] + d]);
        }
      int ax = 0;
      for (int d = 1; d < 3; ++d)
        if (ch[d] - cl[d] > ch[ax] - cl[ax]) ax = d;
      const int64_t mid = b + (e - b) / 2;
      std::nth_element(idx.begin() + b, idx.begin() + mid, idx.begin() + e, [&](int64_t x, int64_t y) {
        const double cx = cen[3 * x + ax], cy = cen[3 * y + ax];
        return cx < cy || (cx == cy && x < y);
      });
      std::sort(idx.begin() + b, idx.begin() + mid);  // deterministic order inside the halves
      std::sort(idx.begin() + mid, idx.begin() + e);
      std::vector<std::pair<int32_t, int32_t>> bl, br;
      node.left = build(b, mid, bl);
      node.right = build(mid, e, br);
      cancel_into(bl, br);
      boundary.swap(bl);
    }
    SegWriter sw{V, &cap_seg};
    node.cap_begin = (int32_t)cap_seg.size();
    if (!boundary.empty()) cap_strips(boundary, sw);
    node.cap_cnt = (int32_t)cap_seg.size() - node.cap_begin;
    node.cap_tris = (int32_t)sw.tris;
    for (int d = 0; d < 3; ++d) {
      node.lo[d] = lo[d];
      node.hi[d] = hi[d];
    }
    node.skip = (int32_t)nodes->size();  // pre-order: the subtree is [me, skip)
    (*nodes)[me] = node;
    return me;
  }
};

}  // namespace

// Builds the cap tree of one closed surface: appends its nodes (indices from
// node_base), its segment block (entries from seg_base: the leaves'
// segments, leaf_entries of them, then the caps') and its triangle indices
// in leaf order (positions from tidx_base; a leaf's triangles are
// tidx[tri_begin .. tri_begin + leaf_tris)).
void build_cap_tree(const float *V, const int32_t *T, int64_t nt, int64_t node_base, int64_t seg_base,
                    int64_t tidx_base, std::vector<CapNode> &nodes, std::vector<Entry> &seg,
                    std::vector<int32_t> &tidx, int32_t *root, int64_t *leaf_entries) {
  Builder bd;
  bd.V = V;
  bd.T = T;
  std::vector<CapNode> local;
  bd.nodes = &local;
  bd.idx.resize((size_t)nt);
  bd.cen.resize((size_t)nt * 3);
  for (int64_t t = 0; t < nt; ++t) {
    bd.idx[(size_t)t] = t;
    for (int d = 0; d < 3; ++d)
      bd.cen[3 * t + d] = ((double)V[3 * (int64_t)T[3 * t] + d] + V[3 * (int64_t)T[3 * t + 1] + d] +
                           V[3 * (int64_t)T[3 * t + 2] + d]) / 3.0;
  }
  std::vector<std::pair<int32_t, int32_t>> boundary;
  if (nt > 0) bd.build(0, nt, boundary);
  const int64_t nleaf = (int64_t)bd.leaf_seg.size();
  for (CapNode &n : local) {
    if (n.left >= 0) {
      n.left += (int32_t)node_base;
      n.right += (int32_t)node_base;
    }
    n.leaf_begin += (int32_t)seg_base;
    n.cap_begin += (int32_t)(seg_base + nleaf);
    n.tri_begin += (int32_t)tidx_base;
    n.skip += (int32_t)node_base;
  }
  for (int64_t t : bd.idx) tidx.push_back((int32_t)t);
  *root = (int32_t)node_base;
  *leaf_entries = nleaf;
  nodes.insert(nodes.end(), local.begin(), local.end());
  seg.insert(seg.end(), bd.leaf_seg.begin(), bd.leaf_seg.end());
  seg.insert(seg.end(), bd.cap_seg.begin(), bd.cap_seg.end());
}

}  // namespace zef
