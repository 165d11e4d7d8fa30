// zef_tree.cpp -- exact far-field replacement of surface patches by caps.
//
// A compartment's triangles are split recursively (median of the triangle
// centroids along the longest axis of their box) into a binary tree of
// patches down to leaves of at most kCapLeaf triangles.  Every patch P other
// than the whole (closed) surface has a boundary: the directed edges u -> v
// of its triangles whose opposite v -> u belongs to no triangle of P.  Its
// cap is the fan of triangles (u, v, a) over those edges around an apex a
// (the mean of the boundary vertices); the cap has the same boundary as P,
// so P together with the reversed cap is a closed surface, whose winding
// number is 0 at every point outside its box.  There the solid angle of P
// equals the solid angle of the cap exactly (Sec. 2.1.3: Omega of a closed
// surface is 4 pi times the winding number).  A point tile whose box misses
// the box of P and a therefore sums P's cap instead of P's triangles.
//
// Layout: every compartment's triangles are stored leaf by leaf in tree
// order, followed by the caps of all its nodes; a triangle is four float4
// (A with w = kappa |n|, B, C, n = (B - A) x (C - A) computed in double).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_set>
#include <vector>

#include "zef_internal.h"

namespace zef {

namespace {

inline uint64_t dkey(int32_t u, int32_t v) { return ((uint64_t)(uint32_t)u << 32) | (uint32_t)v; }

struct Builder {
  const float *V;
  const int32_t *T;
  std::vector<CapNode> *nodes;
  std::vector<float4> leaf_tri;  // 4 float4 per triangle, tree order
  std::vector<float4> cap_tri;   // 4 float4 per cap triangle
  std::vector<int64_t> idx;
  std::vector<double> cen;       // 3 per triangle

  void push_tri(std::vector<float4> &out, const double *a, const double *b, const double *c) {
    double e1[3], e2[3];
    for (int q = 0; q < 3; ++q) {
      e1[q] = b[q] - a[q];
      e2[q] = c[q] - a[q];
    }
    const double nx = e1[1] * e2[2] - e1[2] * e2[1];
    const double ny = e1[2] * e2[0] - e1[0] * e2[2];
    const double nz = e1[0] * e2[1] - e1[1] * e2[0];
    const double nn = std::sqrt(nx * nx + ny * ny + nz * nz);
    out.push_back(make_float4((float)a[0], (float)a[1], (float)a[2], (float)(kKappa * nn)));
    out.push_back(make_float4((float)b[0], (float)b[1], (float)b[2], 0.f));
    out.push_back(make_float4((float)c[0], (float)c[1], (float)c[2], 0.f));
    out.push_back(make_float4((float)nx, (float)ny, (float)nz, 0.f));
  }

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
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t k = b; k < e; ++k)
      for (int q = 0; q < 3; ++q) {
        const float *p = V + 3 * (int64_t)T[3 * idx[k] + q];
        for (int d = 0; d < 3; ++d) {
          lo[d] = std::min(lo[d], (double)p[d]);
          hi[d] = std::max(hi[d], (double)p[d]);
        }
      }
    CapNode node{};
    node.left = node.right = -1;
    if (e - b <= kCapLeaf) {
      node.tri_begin = (int32_t)(leaf_tri.size() / 4);
      node.tri_cnt = (int32_t)(e - b);
      std::vector<std::pair<int32_t, int32_t>> edges;
      for (int64_t k = b; k < e; ++k) {
        const int32_t *t = T + 3 * idx[k];
        double a[3], bb[3], c[3];
        for (int d = 0; d < 3; ++d) {
          a[d] = V[3 * (int64_t)t[0] + d];
          bb[d] = V[3 * (int64_t)t[1] + d];
          c[d] = V[3 * (int64_t)t[2] + d];
        }
        push_tri(leaf_tri, a, bb, c);
        edges.push_back({t[0], t[1]});
        edges.push_back({t[1], t[2]});
        edges.push_back({t[2], t[0]});
      }
      boundary.clear();
      cancel_into(boundary, edges);
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
    // cap: fan (u, v, apex) over the boundary edges u -> v
    node.cap_begin = (int32_t)(cap_tri.size() / 4);
    node.cap_cnt = (int32_t)boundary.size();
    if (!boundary.empty()) {
      std::vector<int32_t> bv;
      for (auto &ed : boundary) {
        bv.push_back(ed.first);
        bv.push_back(ed.second);
      }
      std::sort(bv.begin(), bv.end());
      bv.erase(std::unique(bv.begin(), bv.end()), bv.end());
      double apex[3] = {0, 0, 0};
      for (int32_t v : bv)
        for (int d = 0; d < 3; ++d) apex[d] += V[3 * (int64_t)v + d];
      for (int d = 0; d < 3; ++d) {
        apex[d] /= (double)bv.size();
        // the fan's vertex is stored in float: bound the box by the stored value
        const double af = (double)(float)apex[d];
        lo[d] = std::min(lo[d], af);
        hi[d] = std::max(hi[d], af);
      }
      for (auto &ed : boundary) {
        double u[3], v[3], a[3];
        for (int d = 0; d < 3; ++d) {
          u[d] = V[3 * (int64_t)ed.first + d];
          v[d] = V[3 * (int64_t)ed.second + d];
          a[d] = (double)(float)apex[d];
        }
        push_tri(cap_tri, u, v, a);
      }
    }
    for (int d = 0; d < 3; ++d) {
      node.lo[d] = (float)lo[d];
      node.hi[d] = (float)hi[d];
    }
    (*nodes)[me] = node;
    return me;
  }
};

}  // namespace

// Builds the cap tree of one closed surface.  Node indices are relative to
// node_base, triangle indices (in units of 4 float4) relative to tri_base;
// appends the nodes and the compartment's triangle block (leaves, then caps).
void build_cap_tree(const float *V, const int32_t *T, int64_t nt, int64_t node_base, int64_t tri_base,
                    std::vector<CapNode> &nodes, std::vector<float4> &tri, int32_t *root, int64_t *leaf_tris) {
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
  const int64_t nleaf = (int64_t)bd.leaf_tri.size() / 4;
  for (CapNode &n : local) {
    if (n.left >= 0) {
      n.left += (int32_t)node_base;
      n.right += (int32_t)node_base;
    }
    n.tri_begin += (int32_t)tri_base;
    n.cap_begin += (int32_t)(tri_base + nleaf);
  }
  *root = (int32_t)node_base;
  *leaf_tris = nleaf;
  nodes.insert(nodes.end(), local.begin(), local.end());
  tri.insert(tri.end(), bd.leaf_tri.begin(), bd.leaf_tri.end());
  tri.insert(tri.end(), bd.cap_tri.begin(), bd.cap_tri.end());
}

}  // namespace zef
