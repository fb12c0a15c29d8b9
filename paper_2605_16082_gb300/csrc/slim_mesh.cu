// Host-side mesh construction: validation, per-triangle geometry, edge adjacency,
// thread-block tiling, upload to the device (Sec. 1 extruded prismatic mesh,
// Sec. 2.1 column-contiguous structure-of-arrays storage).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "slim_internal.h"

namespace slim {

namespace {
thread_local std::string g_err;
}
void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }
const char* last_error() { return g_err.c_str(); }

template <typename T>
static slim_status upload_vec(slim_mesh* m, const std::vector<T>& v, const T** out) {
  void* p = nullptr;
  size_t n = std::max<size_t>(v.size(), 1) * sizeof(T);
  SLIM_CUDA_TRY(cudaMalloc(&p, n));
  m->allocs.push_back(p);
  if (!v.empty()) SLIM_CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = static_cast<const T*>(p);
  return SLIM_OK;
}

static void free_mesh(slim_mesh* m) {
  if (!m) return;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

}  // namespace slim

using namespace slim;

extern "C" const char* slim_last_error(void) { return slim::last_error(); }

extern "C" const char* slim_status_string(slim_status s) {
  switch (s) {
    case SLIM_OK: return "ok";
    case SLIM_ERR_ARG: return "invalid argument";
    case SLIM_ERR_MESH: return "inconsistent mesh";
    case SLIM_ERR_CUDA: return "CUDA error";
    case SLIM_ERR_OOM: return "out of device memory";
    case SLIM_ERR_NONFINITE: return "non-finite value";
    case SLIM_ERR_CFL: return "time step above stability estimate";
    case SLIM_ERR_BOUNDS: return "index out of range";
    case SLIM_ERR_TIMEOUT: return "device wait timed out";
    case SLIM_ERR_UNSUPPORTED: return "unsupported combination";
  }
  return "unknown status";
}

namespace {
slim_status mesh_create(const double* xy, int n_vert, const int* tri, int n_tri, const double* h_tri,
                        const int* n_layers, const double* levels, int n_levels, const signed char* bnd,
                        int tile_prisms, const signed char* tri_class, slim_mesh** out);
}

extern "C" slim_status slim_mesh_create(const double* xy, int n_vert, const int* tri, int n_tri,
                                        const double* h_tri, const int* n_layers,
                                        const double* levels, int n_levels,
                                        const signed char* bnd, int tile_prisms,
                                        slim_mesh** out) {
  clear_error();
  return mesh_create(xy, n_vert, tri, n_tri, h_tri, n_layers, levels, n_levels, bnd, tile_prisms, nullptr,
                     out);
}

extern "C" slim_status slim_mesh_create_part(const double* xy, int n_vert, const int* tri, int n_tri,
                                             const double* h_tri, const int* n_layers,
                                             const double* levels, int n_levels,
                                             const signed char* bnd, int tile_prisms,
                                             const signed char* tri_class, slim_mesh** out) {
  clear_error();
  if (!tri_class) { set_error("tri_class is null"); return SLIM_ERR_ARG; }
  for (int t = 0; t < n_tri; ++t) {
    if (tri_class[t] < 0 || tri_class[t] > 2 || (t > 0 && tri_class[t] < tri_class[t - 1])) {
      set_error("tri_class must be non-decreasing in {0, 1, 2}");
      return SLIM_ERR_ARG;
    }
  }
  return mesh_create(xy, n_vert, tri, n_tri, h_tri, n_layers, levels, n_levels, bnd, tile_prisms, tri_class,
                     out);
}

namespace {
slim_status mesh_create(const double* xy, int n_vert, const int* tri, int n_tri, const double* h_tri,
                        const int* n_layers, const double* levels, int n_levels, const signed char* bnd,
                        int tile_prisms, const signed char* tri_class, slim_mesh** out) {
  if (!out) { set_error("out is null"); return SLIM_ERR_ARG; }
  *out = nullptr;
  if (!xy || !tri || !h_tri || !n_layers || !bnd || n_vert < 3 || n_tri < 1) {
    set_error("null array or empty mesh");
    return SLIM_ERR_ARG;
  }
  if (levels && n_levels < 2) { set_error("levels needs at least 2 entries"); return SLIM_ERR_ARG; }
  if (tile_prisms <= 0) tile_prisms = 256;
  if (tile_prisms != 128 && tile_prisms != 256 && tile_prisms != 512) {
    set_error("tile_prisms must be 128, 256 or 512");
    return SLIM_ERR_ARG;
  }
  const int nt = n_tri;
  std::vector<int> col_off(nt + 1, 0);
  int max_layers = 0;
  for (int t = 0; t < nt; ++t) {
    int N = n_layers[t];
    if (N < 1 || N > SLIM_MAX_LAYERS || N > tile_prisms) {
      set_error("layer count out of range at triangle " + std::to_string(t));
      return SLIM_ERR_ARG;
    }
    if (levels && N > n_levels - 1 + 1) {
      set_error("more layers than levels at triangle " + std::to_string(t));
      return SLIM_ERR_ARG;
    }
    max_layers = std::max(max_layers, N);
    long long next = (long long)col_off[t] + N;
    if (next > (1LL << 30)) { set_error("too many prisms"); return SLIM_ERR_ARG; }
    col_off[t + 1] = (int)next;
  }
  const int P = col_off[nt];
  std::vector<double> jh(nt), gx(3 * nt), gy(3 * nt), enx(3 * nt), eny(3 * nt), elen(3 * nt),
      rin(nt), h(3 * nt);
  for (int t = 0; t < nt; ++t) {
    int v[3];
    for (int a = 0; a < 3; ++a) {
      v[a] = tri[3 * t + a];
      if (v[a] < 0 || v[a] >= n_vert) { set_error("vertex index out of range"); return SLIM_ERR_ARG; }
      double d = h_tri[3 * t + a];
      if (!(d > 0.0) || !std::isfinite(d)) { set_error("depth must be positive"); return SLIM_ERR_ARG; }
      h[a * nt + t] = d;
    }
    double x0 = xy[2 * v[0]], y0 = xy[2 * v[0] + 1];
    double x1 = xy[2 * v[1]], y1 = xy[2 * v[1] + 1];
    double x2 = xy[2 * v[2]], y2 = xy[2 * v[2] + 1];
    double J = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
    if (!(J > 0.0)) {
      set_error("triangle " + std::to_string(t) + " is not counter-clockwise");
      return SLIM_ERR_MESH;
    }
    jh[t] = J;
    // grad phi_1 = (y2 - y0, -(x2 - x0)) / J, grad phi_2 = (-(y1 - y0), x1 - x0) / J
    double g1x = (y2 - y0) / J, g1y = -(x2 - x0) / J;
    double g2x = -(y1 - y0) / J, g2y = (x1 - x0) / J;
    gx[0 * nt + t] = -g1x - g2x; gy[0 * nt + t] = -g1y - g2y;
    gx[1 * nt + t] = g1x; gy[1 * nt + t] = g1y;
    gx[2 * nt + t] = g2x; gy[2 * nt + t] = g2y;
    double per = 0.0;
    for (int e = 0; e < 3; ++e) {
      int a = v[e], b = v[(e + 1) % 3];
      double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
      double L = std::sqrt(dx * dx + dy * dy);
      elen[e * nt + t] = L;
      enx[e * nt + t] = dy / L;
      eny[e * nt + t] = -dx / L;
      per += L;
    }
    rin[t] = J / per;  // area / semi-perimeter
  }
  // adjacency: sort undirected edges
  std::vector<std::pair<long long, int>> edges(3 * (size_t)nt);
  for (int t = 0; t < nt; ++t)
    for (int e = 0; e < 3; ++e) {
      long long a = tri[3 * t + e], b = tri[3 * t + (e + 1) % 3];
      long long lo = std::min(a, b), hi = std::max(a, b);
      edges[3 * t + e] = {lo * (long long)(n_vert + 1) + hi, 3 * t + e};
    }
  std::sort(edges.begin(), edges.end());
  std::vector<int> nbr(3 * nt, -1), nloc(3 * nt, 0);
  for (size_t i = 0; i < edges.size();) {
    size_t j = i;
    while (j < edges.size() && edges[j].first == edges[i].first) ++j;
    if (j - i > 2) { set_error("edge shared by more than two triangles"); return SLIM_ERR_MESH; }
    if (j - i == 2) {
      int te[2] = {edges[i].second, edges[i + 1].second};
      for (int s = 0; s < 2; ++s) {
        int t = te[s] / 3, e = te[s] % 3;
        int tn = te[1 - s] / 3;
        if (bnd[3 * t + e] != 0) {
          set_error("interior edge tagged as boundary at triangle " + std::to_string(t));
          return SLIM_ERR_MESH;
        }
        nbr[e * nt + t] = tn;
        int l[2];
        for (int jj = 0; jj < 2; ++jj) {
          int gv = tri[3 * t + (e + jj) % 3];
          l[jj] = -1;
          for (int a = 0; a < 3; ++a)
            if (tri[3 * tn + a] == gv) l[jj] = a;
          if (l[jj] < 0) { set_error("adjacency mismatch"); return SLIM_ERR_MESH; }
        }
        nloc[e * nt + t] = l[0] | (l[1] << 2);
      }
    } else {
      int t = edges[i].second / 3, e = edges[i].second % 3;
      nbr[e * nt + t] = (bnd[3 * t + e] == 2) ? -2 : -1;
    }
    i = j;
  }
  // tiling: consecutive triangles, at most tile_prisms prisms per tile; a new tile
  // also starts where the triangle class changes (partition meshes)
  std::vector<int> tile_t0;
  tile_t0.push_back(0);
  int class_tile[4] = {0, 0, 0, 0};  // first tile of classes 0, 1, 2 and the end
  int cur = 0;
  for (int t = 0; t < nt; ++t) {
    int N = n_layers[t];
    const bool new_class = tri_class && t > 0 && tri_class[t] != tri_class[t - 1];
    if (cur + N > tile_prisms || (new_class && cur > 0)) {
      tile_t0.push_back(t);
      cur = 0;
    }
    if (tri_class && (t == 0 || tri_class[t] != tri_class[t - 1]))
      for (int c = (t == 0 ? 0 : tri_class[t - 1] + 1); c <= tri_class[t]; ++c)
        class_tile[c] = (int)tile_t0.size() - 1;
    cur += N;
  }
  tile_t0.push_back(nt);
  {
    const int n_tiles = (int)tile_t0.size() - 1;
    const int last = tri_class ? tri_class[nt - 1] : 2;
    for (int c = last + 1; c <= 3; ++c) class_tile[c] = n_tiles;
    if (!tri_class) { class_tile[0] = class_tile[1] = class_tile[2] = 0; class_tile[3] = n_tiles; }
  }
  int max_tile_tris = 0;
  std::vector<int4> tile_info(tile_t0.size() - 1);
  for (size_t i = 0; i + 1 < tile_t0.size(); ++i) {
    const int a = tile_t0[i], b = tile_t0[i + 1];
    max_tile_tris = std::max(max_tile_tris, b - a);
    tile_info[i] = make_int4(a, b - a, col_off[a], col_off[b] - col_off[a]);
  }
  std::vector<int4> einfo(3 * (size_t)nt);
  for (int e = 0; e < 3; ++e)
    for (int t = 0; t < nt; ++t) {
      const int nb = nbr[e * nt + t];
      einfo[e * nt + t] = nb >= 0 ? make_int4(nb, col_off[nb], col_off[nb + 1] - col_off[nb], nloc[e * nt + t])
                                  : make_int4(nb, 0, 0, 0);
    }
  // horizontal interior-penalty length per edge: 1 / min(r_in^-, r_in^+), 0 off interior edges
  std::vector<double> esig(3 * (size_t)nt, 0.0);
  for (int e = 0; e < 3; ++e)
    for (int t = 0; t < nt; ++t) {
      const int nb = nbr[e * nt + t];
      if (nb >= 0) esig[e * nt + t] = 1.0 / std::min(rin[t], rin[nb]);
    }
  std::vector<float> esigf(esig.begin(), esig.end());
  std::vector<double> lev;
  if (levels) lev.assign(levels, levels + n_levels);
  std::vector<double> hN(3 * nt), ih(3 * nt);
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) {
      hN[a * nt + t] = h[a * nt + t] / n_layers[t];
      ih[a * nt + t] = 1.0 / h[a * nt + t];
    }
  std::vector<float> hNf(hN.begin(), hN.end()), ihf(ih.begin(), ih.end()), hf(h.begin(), h.end()),
      levf(lev.begin(), lev.end());

  slim_mesh* m = new slim_mesh();
  m->tile_prisms = tile_prisms;
  DevMesh& d = m->d;
  d.n_tri = nt;
  d.P = P;
  d.n_tiles = (int)tile_t0.size() - 1;
  d.max_layers = max_layers;
  d.max_tile_tris = max_tile_tris;
  d.n_levels = levels ? n_levels : 0;
  std::vector<float> rinf(rin.begin(), rin.end());
  std::vector<float> jhf(jh.begin(), jh.end()), gxf(gx.begin(), gx.end()), gyf(gy.begin(), gy.end()),
      enxf(enx.begin(), enx.end()), enyf(eny.begin(), eny.end()), elenf(elen.begin(), elen.end());
  slim_status st;
#define UP(vec, field)                                   \
  if ((st = upload_vec(m, vec, &d.field)) != SLIM_OK) { \
    free_mesh(m);                                        \
    return st;                                           \
  }
  UP(col_off, col_off);
  UP(tile_t0, tile_t0);
  UP(tile_info, tile_info);
  UP(einfo, einfo);
  UP(jh, jh);
  UP(gx, gx);
  UP(gy, gy);
  UP(enx, enx);
  UP(eny, eny);
  UP(elen, elen);
  UP(rin, rin);
  UP(rinf, rin_f);
  UP(h, h);
  UP(nbr, nbr);
  UP(nloc, nloc);
  UP(lev, levels);
  UP(hN, hN);
  UP(ih, ih);
  UP(hNf, hN_f);
  UP(ihf, ih_f);
  UP(hf, h_f);
  UP(levf, levels_f);
  UP(jhf, jh_f);
  UP(gxf, gx_f);
  UP(gyf, gy_f);
  UP(enxf, enx_f);
  UP(enyf, eny_f);
  UP(elenf, elen_f);
  UP(esig, esig);
  UP(esigf, esig_f);
#undef UP
  if (!levels) { d.levels = nullptr; d.levels_f = nullptr; }
  m->col_off_h = col_off;
  m->tile_t0_h = tile_t0;
  m->nbr_h = nbr;
  for (int c = 0; c < 4; ++c) m->class_tile[c] = class_tile[c];
  *out = m;
  return SLIM_OK;
}
}  // namespace

extern "C" void slim_mesh_destroy(slim_mesh* m) { free_mesh(m); }

extern "C" slim_status slim_mesh_info(const slim_mesh* m, int64_t* n_prisms, int* n_tri,
                                      int* max_layers, int* n_tiles) {
  if (!m) { set_error("mesh is null"); return SLIM_ERR_ARG; }
  if (n_prisms) *n_prisms = m->d.P;
  if (n_tri) *n_tri = m->d.n_tri;
  if (max_layers) *max_layers = m->d.max_layers;
  if (n_tiles) *n_tiles = m->d.n_tiles;
  return SLIM_OK;
}
