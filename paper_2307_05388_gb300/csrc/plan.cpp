// Symbolic phase: nested dissection, elimination tree, fronts, index maps.
// See plan.h for the ordering rules.
#include "plan.h"

#include <algorithm>
#include <cstdio>
#include <functional>

namespace fdfd {

namespace {

struct Rect {
  int x0, x1, y0, y1;  // [x0, x1) x [y0, y1)
  int w() const { return x1 - x0; }
  int h() const { return y1 - y0; }
  long long area() const { return (long long)w() * h(); }
  bool empty() const { return x1 <= x0 || y1 <= y0; }
};

struct Node {
  Rect r;
  std::vector<int> piv;   // grid cells eliminated at this node
  std::vector<int> kids;
  int parent = -1;
};

struct Builder {
  int nx, ny, bx0, by0, bw, bh, leaf;
  std::vector<Node> nodes;

  bool has_box() const { return bw > 0 && bh > 0; }
  bool intersects_box(const Rect& r) const {
    return has_box() && r.x0 < bx0 + bw && r.x1 > bx0 && r.y0 < by0 + bh && r.y1 > by0;
  }
  bool inside_box(const Rect& r) const {
    return has_box() && r.x0 >= bx0 && r.x1 <= bx0 + bw && r.y0 >= by0 && r.y1 <= by0 + bh;
  }
  bool straddles(const Rect& r) const { return intersects_box(r) && !inside_box(r); }

  int build(const Rect& r) {
    if (r.empty()) return -1;
    int id = (int)nodes.size();
    nodes.push_back(Node{});
    nodes[id].r = r;
    bool strad = straddles(r);
    if (!strad && r.area() <= leaf) {
      for (int i = r.x0; i < r.x1; ++i)
        for (int j = r.y0; j < r.y1; ++j) nodes[id].piv.push_back(i * ny + j);
      return id;
    }
    // choose the separator line: axis 0 = a column x = s, axis 1 = a row y = s
    // A straddling rectangle is cut on a box line when that cut is reasonably
    // balanced (each side at least a quarter of the rectangle) or when the
    // rectangle is already leaf-sized; otherwise it is cut in the middle and
    // the box line is taken further down, where it is balanced.
    int axis = -1, s = -1;
    if (strad) {
      double best = -1;
      auto consider = [&](int ax, int line) {
        int lo = ax == 0 ? r.x0 : r.y0, hi = ax == 0 ? r.x1 : r.y1;
        if (line < lo || line >= hi) return;
        double frac = std::min(line - lo, hi - line - 1) / (double)(hi - lo);
        if (frac > best) { best = frac; axis = ax; s = line; }
      };
      consider(0, bx0 - 1);
      consider(0, bx0 + bw);
      consider(1, by0 - 1);
      consider(1, by0 + bh);
      if (best < 0.25 && r.area() > leaf) axis = -1;
    }
    if (axis < 0) {
      if (r.w() >= r.h()) { axis = 0; s = r.x0 + r.w() / 2; }
      else { axis = 1; s = r.y0 + r.h() / 2; }
    }
    Rect a = r, b = r;
    if (axis == 0) {
      for (int j = r.y0; j < r.y1; ++j) nodes[id].piv.push_back(s * ny + j);
      a.x1 = s; b.x0 = s + 1;
    } else {
      for (int i = r.x0; i < r.x1; ++i) nodes[id].piv.push_back(i * ny + s);
      a.y1 = s; b.y0 = s + 1;
    }
    int ca = build(a);
    int cb = build(b);
    if (ca >= 0) { nodes[id].kids.push_back(ca); nodes[ca].parent = id; }
    if (cb >= 0) { nodes[id].kids.push_back(cb); nodes[cb].parent = id; }
    return id;
  }
};

inline long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

}  // namespace

std::string build_plan(int nx, int ny, int bx0, int by0, int bw, int bh, int leaf_area, Plan* out) {
  if (nx <= 0 || ny <= 0) return "grid dimensions must be positive";
  if ((long long)nx * ny * 5 >= (1LL << 31)) return "grid too large for 32-bit entry codes";
  if (bw < 0 || bh < 0 || (bw > 0 && bh > 0 && (bx0 < 0 || by0 < 0 || bx0 + bw > nx || by0 + bh > ny)))
    return "design box outside the grid";
  if (leaf_area < 1) leaf_area = 1;
  Plan& p = *out;
  p = Plan{};
  p.nx = nx; p.ny = ny; p.bx0 = bx0; p.by0 = by0; p.bw = bw; p.bh = bh; p.leaf_area = leaf_area;

  Builder B{nx, ny, bx0, by0, bw, bh, leaf_area, {}};
  B.nodes.reserve((size_t)(2LL * nx * ny / std::max(1, leaf_area) + 64));
  int root = B.build(Rect{0, nx, 0, ny});
  (void)root;

  // postorder (children before parents), iterative to bound stack depth
  const int nn = (int)B.nodes.size();
  std::vector<int> order;
  order.reserve(nn);
  {
    std::vector<std::pair<int, int>> st;
    st.push_back({0, 0});
    while (!st.empty()) {
      auto& t = st.back();
      const Node& nd = B.nodes[t.first];
      if (t.second < (int)nd.kids.size()) {
        int c = nd.kids[t.second++];
        st.push_back({c, 0});
      } else {
        order.push_back(t.first);
        st.pop_back();
      }
    }
  }
  std::vector<int> newid(nn);
  for (int f = 0; f < nn; ++f) newid[order[f]] = f;

  // elimination positions
  p.pos.assign((size_t)nx * ny, -1);
  int cur = 0;
  for (int f = 0; f < nn; ++f) {
    auto& piv = B.nodes[order[f]].piv;
    std::sort(piv.begin(), piv.end());
    for (int c : piv) p.pos[c] = cur++;
  }
  if (cur != nx * ny) return "nested dissection did not cover the grid";

  // fronts
  p.fronts.resize(nn);
  std::vector<std::vector<int>> bnd(nn);
  for (int f = 0; f < nn; ++f) {
    const Node& nd = B.nodes[order[f]];
    const Rect& r = nd.r;
    std::vector<int>& b = bnd[f];
    if (r.x0 > 0) for (int j = r.y0; j < r.y1; ++j) b.push_back((r.x0 - 1) * ny + j);
    if (r.x1 < nx) for (int j = r.y0; j < r.y1; ++j) b.push_back(r.x1 * ny + j);
    if (r.y0 > 0) for (int i = r.x0; i < r.x1; ++i) b.push_back(i * ny + r.y0 - 1);
    if (r.y1 < ny) for (int i = r.x0; i < r.x1; ++i) b.push_back(i * ny + r.y1);
    std::sort(b.begin(), b.end(), [&](int a, int c) { return p.pos[a] < p.pos[c]; });
    FrontDesc& d = p.fronts[f];
    d = FrontDesc{};
    d.k = (int)nd.piv.size();
    d.m = (int)b.size();
    d.n = d.k + d.m;
    d.ld = (int)round_up(d.n, 4);
    d.parent = nd.parent < 0 ? -1 : newid[nd.parent];
  }
  // children lists (in postorder of the children) and levels
  for (int f = 0; f < nn; ++f) {
    const Node& nd = B.nodes[order[f]];
    FrontDesc& d = p.fronts[f];
    d.child0 = (int)p.children.size();
    std::vector<int> kids;
    for (int c : nd.kids) kids.push_back(newid[c]);
    std::sort(kids.begin(), kids.end());
    for (int c : kids) p.children.push_back(c);
    d.nchild = (int)kids.size();
    int lv = 0;
    for (int c : kids) lv = std::max(lv, p.fronts[c].level + 1);
    d.level = lv;
  }
  // index lists, offsets
  long long st = 0, vo = 0, iv = 0;
  int io = 0, po = 0;
  for (int f = 0; f < nn; ++f) {
    FrontDesc& d = p.fronts[f];
    const Node& nd = B.nodes[order[f]];
    d.ldk = (int)round_up(d.k, 4);
    d.iv_off = iv;
    iv += round_up((long long)d.k * d.ldk, 64);
    d.idx_off = io;
    for (int c : nd.piv) p.idx.push_back(c);
    for (int c : bnd[f]) p.idx.push_back(c);
    io += d.n;
    d.st_off = st;
    st += round_up((long long)d.n * d.ld, 64);
    d.v_off = vo;
    vo += round_up(d.n, 4);
    d.piv_off = po;
    po += d.k;
    p.max_front = std::max(p.max_front, d.n);
  }
  p.store_total = st;
  p.inv_total = iv;
  p.vec_total = vo;
  p.perm_total = po;

  // boundary sanity: each boundary cell is eliminated after every pivot of the front
  for (int f = 0; f < nn; ++f) {
    const FrontDesc& d = p.fronts[f];
    int maxp = -1;
    for (int a = 0; a < d.k; ++a) maxp = std::max(maxp, p.pos[p.idx[d.idx_off + a]]);
    for (int t = 0; t < d.m; ++t)
      if (p.pos[p.idx[d.idx_off + d.k + t]] <= maxp) return "boundary variable eliminated before a pivot";
  }

  // extend-add inverse maps: for child f, parent-local index -> f's boundary index
  {
    std::vector<int> loc((size_t)nx * ny, -1);
    for (int f = 0; f < nn; ++f) p.fronts[f].inv_off = -1;
    for (int par = 0; par < nn; ++par) {
      const FrontDesc& pd = p.fronts[par];
      for (int a = 0; a < pd.n; ++a) loc[p.idx[pd.idx_off + a]] = a;
      for (int ci = 0; ci < pd.nchild; ++ci) {
        int c = p.children[pd.child0 + ci];
        FrontDesc& cd = p.fronts[c];
        cd.inv_off = (int)p.inv.size();
        p.inv.resize(p.inv.size() + pd.n, -1);
        for (int t = 0; t < cd.m; ++t) {
          int cell = p.idx[cd.idx_off + cd.k + t];
          int a = loc[cell];
          if (a < 0) return "child boundary variable missing from the parent front";
          p.inv[cd.inv_off + a] = t;
        }
      }
      for (int a = 0; a < pd.n; ++a) loc[p.idx[pd.idx_off + a]] = -1;
    }
  }

  // original entries: A[r][c] belongs to the front that eliminates min(pos r, pos c)
  {
    std::vector<int> loc((size_t)nx * ny, -1);
    for (int f = 0; f < nn; ++f) {
      FrontDesc& d = p.fronts[f];
      for (int a = 0; a < d.n; ++a) loc[p.idx[d.idx_off + a]] = a;
      std::vector<std::pair<long long, int>> ent;   // (local row * n + local col, code)
      for (int a = 0; a < d.k; ++a) {
        int cell = p.idx[d.idx_off + a];
        int i = cell / ny, j = cell % ny;
        const int di[5] = {0, -1, 1, 0, 0}, dj[5] = {0, 0, 0, -1, 1};
        const int opp[5] = {DIR_DIAG, DIR_XP, DIR_XM, DIR_YP, DIR_YM};
        for (int dir = 0; dir < 5; ++dir) {
          int ii = i + di[dir], jj = j + dj[dir];
          if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
          int q = ii * ny + jj;
          if (p.pos[q] < p.pos[cell]) continue;          // owned by an earlier front
          int b = loc[q];
          if (b < 0) return "stencil neighbour missing from the front";
          ent.push_back({(long long)a * d.n + b, cell * 5 + dir});
          if (q != cell) ent.push_back({(long long)b * d.n + a, q * 5 + opp[dir]});
        }
      }
      std::sort(ent.begin(), ent.end());
      d.orig_off = (int)p.orig_ptr.size();
      const int base = (int)p.orig_col.size();
      size_t e = 0;
      for (int a = 0; a <= d.n; ++a) {      // orig_ptr values are absolute offsets
        while (e < ent.size() && ent[e].first < (long long)a * d.n) ++e;
        p.orig_ptr.push_back(base + (int)e);
      }
      for (auto& en : ent) {
        p.orig_col.push_back((int)(en.first % d.n));
        p.orig_code.push_back(en.second);
      }
      for (int a = 0; a < d.n; ++a) loc[p.idx[d.idx_off + a]] = -1;
    }
  }

  // design-affected fronts: subtree holds a design pixel
  for (int f = 0; f < nn; ++f) {
    FrontDesc& d = p.fronts[f];
    int des = 0;
    if (bw > 0 && bh > 0)
      for (int a = 0; a < d.k && !des; ++a) {
        int cell = p.idx[d.idx_off + a];
        int i = cell / ny, j = cell % ny;
        if (i >= bx0 && i < bx0 + bw && j >= by0 && j < by0 + bh) des = 1;
      }
    for (int ci = 0; ci < d.nchild && !des; ++ci) des = p.fronts[p.children[d.child0 + ci]].design;
    d.design = des;
  }

  // levels and work model
  for (const auto& d : p.fronts) p.n_levels = std::max(p.n_levels, d.level + 1);
  p.level_fronts.assign(p.n_levels, {});
  for (int f = 0; f < nn; ++f) p.level_fronts[p.fronts[f].level].push_back(f);
  for (const auto& d : p.fronts) {
    double k = d.k, m = d.m;
    double cfma = k * k * k / 3.0 + k * k * m + k * m * m;   // complex multiply-adds
    p.flops_factor += 8.0 * cfma;
    if (d.design) p.flops_design += 8.0 * cfma;
    p.factor_entries += (long long)d.k * d.k + 2LL * d.k * d.m;
  }
  return validate_plan(p);
}

std::string validate_plan(const Plan& p) {
  const int nn = (int)p.fronts.size();
  // every cell is a pivot of exactly one front
  std::vector<int> seen((size_t)p.nx * p.ny, 0);
  for (const auto& d : p.fronts)
    for (int a = 0; a < d.k; ++a) seen[p.idx[d.idx_off + a]]++;
  for (int v : seen) if (v != 1) return "a cell is not a pivot of exactly one front";
  // every stencil entry assembled exactly once
  long long expect = 0;
  for (int i = 0; i < p.nx; ++i)
    for (int j = 0; j < p.ny; ++j)
      expect += 1 + (i > 0) + (i + 1 < p.nx) + (j > 0) + (j + 1 < p.ny);
  if ((long long)p.orig_code.size() != expect) return "original entry count mismatch";
  std::vector<char> hit((size_t)expect > 0 ? (size_t)p.nx * p.ny * 5 : 0, 0);
  for (int c : p.orig_code) {
    if (hit[c]) return "original entry assembled twice";
    hit[c] = 1;
  }
  // extend-add maps injective and within range
  for (int f = 0; f < nn; ++f) {
    const FrontDesc& d = p.fronts[f];
    if (d.parent < 0) continue;
    const FrontDesc& pd = p.fronts[d.parent];
    std::vector<char> used(d.m, 0);
    int cnt = 0;
    for (int a = 0; a < pd.n; ++a) {
      int t = p.inv[d.inv_off + a];
      if (t < 0) continue;
      if (t >= d.m || used[t]) return "extend-add map not injective";
      used[t] = 1;
      ++cnt;
    }
    if (cnt != d.m) return "extend-add map incomplete";
    if (pd.level <= d.level) return "parent level not above child level";
  }
  return "";
}

}  // namespace fdfd
