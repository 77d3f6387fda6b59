// Host topology of unstructured meshes (see utopo.h).
#include "utopo.h"

#include <algorithm>
#include <set>

namespace pmg {

namespace {

uint64_t splitmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// reference entities of a cell: for every edge (and face in 3D) the corners in
// lexicographic order of its running axes (first running axis fastest)
struct RefEntity {
  std::vector<int> run;        // running axes, increasing
  std::vector<int> corners;    // 2 (edge) or 4 (face) corner ids
};

std::vector<RefEntity> ref_entities(int dim, int nrun) {
  std::vector<RefEntity> out;
  std::vector<int> axes(dim);
  for (int i = 0; i < dim; ++i) axes[i] = i;
  // choose `nrun` running axes
  for (int mask = 0; mask < (1 << dim); ++mask) {
    if (__builtin_popcount(mask) != nrun) continue;
    std::vector<int> run, fixed;
    for (int a = 0; a < dim; ++a) ((mask >> a) & 1 ? run : fixed).push_back(a);
    for (int fv = 0; fv < (1 << (int)fixed.size()); ++fv) {
      RefEntity e;
      e.run = run;
      for (int b = 0; b < (1 << nrun); ++b) {
        int c = 0;
        for (size_t i = 0; i < fixed.size(); ++i) c |= ((fv >> i) & 1) << fixed[i];
        for (int i = 0; i < nrun; ++i) c |= ((b >> i) & 1) << run[i];
        e.corners.push_back(c);
      }
      out.push_back(e);
    }
  }
  return out;
}

}  // namespace

std::string utopo_build(int dim, int64_t nv, int64_t nc, const int64_t* cells, const uint8_t* vob, UTopo* t) {
  if (dim != 2 && dim != 3) return "dim must be 2 or 3";
  if (nv < 1 || nc < 1 || !cells) return "empty mesh";
  const int ncorner = 1 << dim;
  t->dim = dim;
  t->nv = nv;
  t->nc = nc;
  t->cells.assign(cells, cells + nc * ncorner);
  for (int64_t v : t->cells)
    if (v < 0 || v >= nv) return "cell vertex id out of range";
  std::map<std::array<int64_t, 2>, std::vector<int64_t>> ecells;
  std::map<std::array<int64_t, 4>, std::vector<int64_t>> fcells;
  const auto E = ref_entities(dim, 1), F = dim == 3 ? ref_entities(3, 2) : std::vector<RefEntity>();
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t* cv = &t->cells[c * ncorner];
    std::set<int64_t> distinct(cv, cv + ncorner);
    if ((int)distinct.size() != ncorner) return "a cell repeats a vertex";
    for (const auto& e : E) {
      std::array<int64_t, 2> k = {cv[e.corners[0]], cv[e.corners[1]]};
      std::sort(k.begin(), k.end());
      ecells[k].push_back(c);
    }
    for (const auto& f : F) {
      std::array<int64_t, 4> k = {cv[f.corners[0]], cv[f.corners[1]], cv[f.corners[2]], cv[f.corners[3]]};
      std::sort(k.begin(), k.end());
      fcells[k].push_back(c);
    }
  }
  t->edges.clear();
  t->edge_id.clear();
  for (const auto& kv : ecells) {
    t->edge_id[kv.first] = (int64_t)t->edges.size();
    t->edges.push_back(kv.first);
  }
  t->faces.clear();
  t->face_id.clear();
  for (const auto& kv : fcells) {
    t->face_id[kv.first] = (int64_t)t->faces.size();
    t->faces.push_back(kv.first);
  }
  t->vertex_cells.assign(nv, {});
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < ncorner; ++k) t->vertex_cells[t->cells[c * ncorner + k]].push_back(c);
  for (auto& vc : t->vertex_cells) {
    std::sort(vc.begin(), vc.end());
    vc.erase(std::unique(vc.begin(), vc.end()), vc.end());
    if (vc.empty()) return "a vertex belongs to no cell";
  }
  // boundary: facets of one cell
  t->edge_on_boundary.assign(t->edges.size(), 0);
  t->face_on_boundary.assign(t->faces.size(), 0);
  std::vector<uint8_t> vb(nv, 0);
  if (dim == 2) {
    for (const auto& kv : ecells) {
      if (kv.second.size() > 2) return "an edge is shared by more than two cells";
      if (kv.second.size() == 1) {
        t->edge_on_boundary[t->edge_id[kv.first]] = 1;
        vb[kv.first[0]] = vb[kv.first[1]] = 1;
      }
    }
  } else {
    for (const auto& kv : fcells) {
      if (kv.second.size() > 2) return "a face is shared by more than two cells";
      if (kv.second.size() != 1) continue;
      t->face_on_boundary[t->face_id[kv.first]] = 1;
      // the face's corners and edges, from the cell that holds it
      const int64_t c = kv.second[0];
      const int64_t* cv = &t->cells[c * ncorner];
      for (const auto& f : F) {
        std::array<int64_t, 4> k = {cv[f.corners[0]], cv[f.corners[1]], cv[f.corners[2]], cv[f.corners[3]]};
        std::sort(k.begin(), k.end());
        if (k != kv.first) continue;
        for (int i = 0; i < 4; ++i) vb[cv[f.corners[i]]] = 1;
        const int pairs[4][2] = {{0, 1}, {2, 3}, {0, 2}, {1, 3}};
        for (const auto& pr : pairs) {
          std::array<int64_t, 2> ek = {cv[f.corners[pr[0]]], cv[f.corners[pr[1]]]};
          std::sort(ek.begin(), ek.end());
          t->edge_on_boundary[t->edge_id[ek]] = 1;
        }
      }
    }
  }
  if (vob) {
    t->vertex_on_boundary.assign(vob, vob + nv);
    for (int64_t v = 0; v < nv; ++v)
      if (vb[v] && !vob[v]) return "vertex_on_boundary misses a vertex of a boundary facet";
  } else {
    t->vertex_on_boundary = vb;
  }
  return "";
}

int64_t utopo_ndofs(const UTopo& t, int q) {
  const int64_t m = q - 1;
  return t.nv + (int64_t)t.edges.size() * m + (int64_t)t.faces.size() * m * m + t.nc * (t.dim == 3 ? m * m * m : m * m);
}

std::vector<int32_t> utopo_cell_dofs(const UTopo& t, int q) {
  const int d = t.dim, n = q + 1, ncorner = 1 << d;
  int nloc = 1;
  for (int k = 0; k < d; ++k) nloc *= n;
  const int64_t m = q - 1;
  const int64_t e0 = t.nv, f0 = e0 + (int64_t)t.edges.size() * m, c0 = f0 + (int64_t)t.faces.size() * m * m;
  const int64_t mint = d == 3 ? m * m * m : m * m;
  std::vector<int32_t> out((size_t)t.nc * nloc);
  for (int64_t c = 0; c < t.nc; ++c) {
    const int64_t* cv = &t.cells[c * ncorner];
    for (int li = 0; li < nloc; ++li) {
      int mi[3] = {0, 0, 0}, rem = li;
      for (int k = 0; k < d; ++k) { mi[k] = rem % n; rem /= n; }
      int onb = 0, run[3], nrun = 0, fixedbits = 0;
      for (int k = 0; k < d; ++k) {
        if (mi[k] == 0 || mi[k] == q) {
          ++onb;
          fixedbits |= (mi[k] == q ? 1 : 0) << k;
        } else {
          run[nrun++] = k;
        }
      }
      int64_t g;
      if (nrun == 0) {                                          // a vertex
        g = cv[fixedbits];
      } else if (nrun == 1) {                                   // an edge
        const int a = run[0];
        const int64_t v0 = cv[fixedbits], v1 = cv[fixedbits | (1 << a)];
        const int tpos = v0 < v1 ? mi[a] : q - mi[a];
        std::array<int64_t, 2> k = {std::min(v0, v1), std::max(v0, v1)};
        g = e0 + t.edge_id.at(k) * m + (tpos - 1);
      } else if (nrun == 2 && d == 3) {                         // a face
        const int r1 = run[0], r2 = run[1];
        int64_t ids[2][2];
        for (int b1 = 0; b1 < 2; ++b1)
          for (int b2 = 0; b2 < 2; ++b2) ids[b1][b2] = cv[fixedbits | (b1 << r1) | (b2 << r2)];
        int a1 = 0, a2 = 0;
        for (int b1 = 0; b1 < 2; ++b1)
          for (int b2 = 0; b2 < 2; ++b2)
            if (ids[b1][b2] < ids[a1][a2]) { a1 = b1; a2 = b2; }
        const int64_t n1 = ids[1 - a1][a2], n2 = ids[a1][1 - a2];   // anchor's neighbours along r1, r2
        const int s1 = a1 == 0 ? mi[r1] : q - mi[r1];
        const int s2 = a2 == 0 ? mi[r2] : q - mi[r2];
        const int u = n1 < n2 ? s1 : s2, w = n1 < n2 ? s2 : s1;
        std::array<int64_t, 4> k = {ids[0][0], ids[0][1], ids[1][0], ids[1][1]};
        std::sort(k.begin(), k.end());
        g = f0 + t.face_id.at(k) * m * m + (u - 1) + m * (w - 1);
      } else {                                                  // cell interior
        int64_t loc = 0, mul = 1;
        for (int k = 0; k < d; ++k) { loc += (mi[k] - 1) * mul; mul *= m; }
        g = c0 + c * mint + loc;
      }
      out[(size_t)c * nloc + li] = (int32_t)g;
    }
  }
  return out;
}

std::vector<uint8_t> utopo_boundary_dofs(const UTopo& t, int q) {
  const int64_t m = q - 1;
  std::vector<uint8_t> out((size_t)utopo_ndofs(t, q), 0);
  for (int64_t v = 0; v < t.nv; ++v) out[v] = t.vertex_on_boundary[v];
  const int64_t e0 = t.nv, f0 = e0 + (int64_t)t.edges.size() * m;
  for (size_t e = 0; e < t.edges.size(); ++e)
    if (t.edge_on_boundary[e])
      for (int64_t i = 0; i < m; ++i) out[e0 + e * m + i] = 1;
  for (size_t f = 0; f < t.faces.size(); ++f)
    if (t.face_on_boundary[f])
      for (int64_t i = 0; i < m * m; ++i) out[f0 + f * m * m + i] = 1;
  return out;
}

std::vector<int64_t> utopo_patch_vertices(const UTopo& t) {
  std::vector<int64_t> out;
  for (int64_t v = 0; v < t.nv; ++v)
    if (!t.vertex_on_boundary[v] && !t.vertex_cells[v].empty()) out.push_back(v);
  return out;
}

std::vector<uint8_t> utopo_colours(const UTopo& t, const std::vector<int64_t>& pverts, uint64_t seed, int* ncolours) {
  const int ncorner = 1 << t.dim;
  std::vector<int64_t> order(pverts);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const uint64_t ka = splitmix64((uint64_t)a ^ seed), kb = splitmix64((uint64_t)b ^ seed);
    return ka != kb ? ka > kb : a > b;                     // decreasing (priority, id)
  });
  std::vector<int> col(t.nv, -1);
  int nmax = 0;
  for (int64_t v : order) {
    std::vector<char> used(256, 0);
    for (int64_t c : t.vertex_cells[v])
      for (int k = 0; k < ncorner; ++k) {
        const int cw = col[t.cells[c * ncorner + k]];
        if (cw >= 0) used[cw] = 1;
      }
    int k = 0;
    while (k < 255 && used[k]) ++k;
    col[v] = k;
    nmax = std::max(nmax, k + 1);
  }
  std::vector<uint8_t> out(pverts.size());
  for (size_t i = 0; i < pverts.size(); ++i) out[i] = (uint8_t)col[pverts[i]];
  *ncolours = nmax;
  return out;
}

}  // namespace pmg
