// bm_mesh.cpp -- host preparation of the finite-volume mesh (once per mesh).
//
// Builds the quantities of Section "Domain discretization" (edge lengths l_ij,
// unit normals n_ij pointing from cell i to cell j, areas |Omega_i|), renumbers
// the cells along a Hilbert curve of their centroids so that neighbours sit close
// in memory, and packs per-tile edge lists for the tiled step kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <sstream>

#include "bm_internal.h"

namespace bm {

namespace {

// Position of (x, y) on the Hilbert curve filling an n x n grid (n a power of 2):
// the classic quadrant-by-quadrant construction, rotating the frame at each level.
uint64_t hilbert_index(uint32_t n, uint32_t x, uint32_t y) {
  uint64_t d = 0;
  for (uint32_t s = n / 2; s > 0; s /= 2) {
    uint32_t rx = (x & s) ? 1u : 0u;
    uint32_t ry = (y & s) ? 1u : 0u;
    d += static_cast<uint64_t>(s) * s * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = n - 1 - x;
        y = n - 1 - y;
      }
      std::swap(x, y);
    }
  }
  return d;
}

struct Half {
  uint64_t key;  // (min node << 32) | max node
  int64_t tk;    // 3 * triangle + local edge
};

}  // namespace

bm_status prepare_mesh(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
                       const double* z, const double* man, const uint8_t* tag, HostMesh* out) {
  if (!xy || !tri || !z || !man || !tag || !out) return fail(BM_EINVAL, "bm_mesh_create: NULL argument");
  if (n_tri < 1) return fail(BM_EINVAL, "bm_mesh_create: n_tri must be >= 1");
  if (n_nodes < 3) return fail(BM_EINVAL, "bm_mesh_create: n_nodes must be >= 3");
  if (n_tri > (int64_t(1) << 30)) return fail(BM_EINVAL, "bm_mesh_create: n_tri too large");
  const int64_t N = n_tri;
  for (int64_t i = 0; i < 2 * n_nodes; ++i)
    if (!std::isfinite(xy[i])) return fail(BM_EINVAL, "bm_mesh_create: non-finite node coordinate");

  // 1. orientation, area, per-edge tags of the (possibly reoriented) triangles
  std::vector<int32_t> v(3 * N);
  std::vector<uint8_t> tg(3 * N);
  std::vector<double> area(N), cx(N), cy(N);
  for (int64_t t = 0; t < N; ++t) {
    int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= n_nodes || b >= n_nodes || c >= n_nodes) {
      std::ostringstream os;
      os << "bm_mesh_create: triangle " << t << " has a node index out of range";
      return fail(BM_EINVAL, os.str());
    }
    if (!std::isfinite(z[t]) || !std::isfinite(man[t]) || man[t] < 0)
      return fail(BM_EINVAL, "bm_mesh_create: z_bed and manning_n must be finite, n >= 0");
    double ax = xy[2 * a], ay = xy[2 * a + 1], bx = xy[2 * b], by = xy[2 * b + 1];
    double qx = xy[2 * c], qy = xy[2 * c + 1];
    double twice = (bx - ax) * (qy - ay) - (qx - ax) * (by - ay);
    if (twice < 0) {  // clockwise: (a, c, b); its edges k are the old edges 2, 1, 0
      v[3 * t] = a; v[3 * t + 1] = c; v[3 * t + 2] = b;
      tg[3 * t] = tag[3 * t + 2]; tg[3 * t + 1] = tag[3 * t + 1]; tg[3 * t + 2] = tag[3 * t];
      twice = -twice;
    } else {
      v[3 * t] = a; v[3 * t + 1] = b; v[3 * t + 2] = c;
      tg[3 * t] = tag[3 * t]; tg[3 * t + 1] = tag[3 * t + 1]; tg[3 * t + 2] = tag[3 * t + 2];
    }
    if (!(twice > 0)) {
      std::ostringstream os;
      os << "bm_mesh_create: triangle " << t << " is degenerate (area <= 0)";
      return fail(BM_EINVAL, os.str());
    }
    area[t] = 0.5 * twice;
    cx[t] = (ax + bx + qx) / 3.0;
    cy[t] = (ay + by + qy) / 3.0;
  }

  // 2. edges: group the 3N half-edges by their node pair
  std::vector<Half> hs(3 * N);
  for (int64_t t = 0; t < N; ++t)
    for (int k = 0; k < 3; ++k) {
      uint64_t p0 = static_cast<uint32_t>(v[3 * t + k]);
      uint64_t p1 = static_cast<uint32_t>(v[3 * t + (k + 1) % 3]);
      hs[3 * t + k].key = p0 < p1 ? (p0 << 32 | p1) : (p1 << 32 | p0);
      hs[3 * t + k].tk = 3 * t + k;
    }
  std::sort(hs.begin(), hs.end(), [](const Half& a, const Half& b) {
    return a.key != b.key ? a.key < b.key : a.tk < b.tk;
  });
  // per undirected edge: left triangle (lower caller index), right triangle or code
  std::vector<int64_t> edge_of(3 * N);  // half-edge tk -> edge id
  std::vector<int64_t> gl, gr;
  std::vector<double> gnx, gny, glen;
  gl.reserve(3 * N / 2 + 16);
  for (int64_t i = 0; i < 3 * N;) {
    int64_t j = i + 1;
    while (j < 3 * N && hs[j].key == hs[i].key) ++j;
    if (j - i > 2) return fail(BM_EINVAL, "bm_mesh_create: an edge is shared by more than two triangles");
    int64_t e = static_cast<int64_t>(gl.size());
    int64_t tkL = hs[i].tk, tL = tkL / 3;
    int kL = static_cast<int>(tkL % 3);
    int32_t p0 = v[tkL], p1 = v[3 * tL + (kL + 1) % 3];
    double dx = xy[2 * p1] - xy[2 * p0], dy = xy[2 * p1 + 1] - xy[2 * p0 + 1];
    double l = std::sqrt(dx * dx + dy * dy);
    edge_of[tkL] = e;
    gl.push_back(tL);
    gnx.push_back(dy / l);  // outward normal of the left triangle's counter-clockwise edge
    gny.push_back(-dx / l);
    glen.push_back(l);
    if (j - i == 2) {
      int64_t tkR = hs[i + 1].tk, tR = tkR / 3;
      int kR = static_cast<int>(tkR % 3);
      int32_t q0 = v[tkR], q1 = v[3 * tR + (kR + 1) % 3];
      if (!(q0 == p1 && q1 == p0))
        return fail(BM_EINVAL, "bm_mesh_create: two triangles traverse an edge in the same direction");
      edge_of[tkR] = e;
      gr.push_back(tR);
    } else {
      uint8_t tt = tg[tkL];
      if (tt > 5) return fail(BM_EINVAL, "bm_mesh_create: boundary edge tag outside {0,1,2,3,4,5}");
      static const int32_t kOfTag[6] = {kWall, kTransmissive, kInflow, kHqTag, kWeirTag, kLevelTag};
      gr.push_back(kOfTag[tt]);
    }
    i = j;
  }
  const int64_t E = static_cast<int64_t>(gl.size());

  // 3. Hilbert renumbering of cells by centroid
  double xmin = cx[0], xmax = cx[0], ymin = cy[0], ymax = cy[0];
  for (int64_t t = 1; t < N; ++t) {
    xmin = std::min(xmin, cx[t]); xmax = std::max(xmax, cx[t]);
    ymin = std::min(ymin, cy[t]); ymax = std::max(ymax, cy[t]);
  }
  double ext = std::max(xmax - xmin, ymax - ymin);
  if (!(ext > 0)) ext = 1.0;
  const uint32_t side = 1u << 16;
  std::vector<std::pair<uint64_t, int32_t>> order(N);
  for (int64_t t = 0; t < N; ++t) {
    uint32_t qx = static_cast<uint32_t>(std::min(65535.0, std::floor((cx[t] - xmin) / ext * 65535.0)));
    uint32_t qy = static_cast<uint32_t>(std::min(65535.0, std::floor((cy[t] - ymin) / ext * 65535.0)));
    order[t] = {hilbert_index(side, qx, qy), static_cast<int32_t>(t)};
  }
  std::sort(order.begin(), order.end());
  HostMesh& m = *out;
  m = HostMesh();
  m.n_cells = N;
  m.n_edges = E;
  m.n_tiles = (N + kTile - 1) / kTile;
  const int64_t Np = m.n_tiles * kTile;
  m.perm.resize(N);
  std::vector<int32_t> newid(N);
  for (int64_t i = 0; i < N; ++i) {
    m.perm[i] = order[i].second;
    newid[order[i].second] = static_cast<int32_t>(i);
  }
  m.z.assign(Np, 0.0);
  m.man.assign(Np, 0.0);
  m.inv_area.assign(Np, 0.0);
  m.area.assign(Np, 0.0);
  m.slots.assign(Np, 0);
  m.z_min = z[0];
  for (int64_t i = 0; i < N; ++i) {
    int32_t t = m.perm[i];
    m.z[i] = z[t];
    m.man[i] = man[t];
    m.area[i] = area[t];
    m.inv_area[i] = 1.0 / area[t];
    m.z_min = std::min(m.z_min, z[t]);
  }

  // 4. boundary lists: the inflow, then the h-Q, then the weir, then the water-level
  // edges; listed edge j is coded kInflow - j
  std::vector<int32_t> code(E);
  for (int64_t e = 0; e < E; ++e) {
    if (gr[e] >= 0) {
      code[e] = newid[gr[e]];
    } else {
      ++m.n_boundary;
      code[e] = static_cast<int32_t>(gr[e]);
    }
  }
  for (int32_t kind : {kInflow, kHqTag, kWeirTag, kLevelTag}) {
    for (int64_t e = 0; e < E; ++e) {
      if (gr[e] != kind) continue;
      code[e] = kInflow - static_cast<int32_t>(m.in_cell.size());
      m.in_cell.push_back(newid[gl[e]]);
      m.in_len.push_back(glen[e]);
      m.in_nx.push_back(gnx[e]);
      m.in_ny.push_back(gny[e]);
      if (kind == kInflow) {
        m.inflow_len += glen[e];
        ++m.n_inflow;
      } else if (kind == kHqTag) {
        ++m.n_hq;
      } else if (kind == kWeirTag) {
        ++m.n_weir;
      } else {
        ++m.n_level;
      }
    }
  }

  // 5. per-tile edge lists and per-cell slots
  std::vector<int64_t> stamp(E, -1);
  std::vector<int32_t> pos(E, 0);
  m.eoff.assign(m.n_tiles + 1, 0);
  m.eL.reserve(E * 2);
  for (int64_t tile = 0; tile < m.n_tiles; ++tile) {
    int32_t cnt = 0;
    bool has_boundary = false;
    m.eoff[tile] = static_cast<int64_t>(m.eL.size());
    for (int64_t i = tile * kTile; i < std::min(N, (tile + 1) * kTile); ++i) {
      int32_t t = m.perm[i];
      uint64_t packed = 0;
      for (int k = 0; k < 3; ++k) {
        int64_t e = edge_of[3 * t + k];
        if (stamp[e] != tile) {
          stamp[e] = tile;
          pos[e] = cnt++;
          m.eL.push_back(newid[gl[e]]);
          m.eR.push_back(code[e]);
          m.enx.push_back(gnx[e]);
          m.eny.push_back(gny[e]);
          m.elen.push_back(glen[e]);
          if (code[e] < 0 && code[e] != kWall) has_boundary = true;  // a wall carries no mass
        }
        uint64_t side_bit = (gl[e] == t) ? 0u : 1u;
        packed |= ((static_cast<uint64_t>(pos[e]) << 1) | side_bit) << (16 * k);
      }
      m.slots[i] = packed;
    }
    if (cnt > kMaxTileEdges) return fail(BM_EINVAL, "bm_mesh_create: internal tile overflow");
    if (has_boundary) m.btiles.push_back(static_cast<int32_t>(tile));
  }
  m.eoff[m.n_tiles] = static_cast<int64_t>(m.eL.size());
  return BM_OK;
}

}  // namespace bm

namespace bm {

namespace {
template <typename T>
void put(std::vector<unsigned char>& d, size_t at, T v) {
  std::memcpy(d.data() + at, &v, sizeof(T));
}

template <typename T>
bm_status build_records_t(const HostMesh& m, TileRecords* out) {
  constexpr int S = sizeof(T);
  using RL = RecLayout<S>;
  TileRecords& r = *out;
  r = TileRecords();
  const int64_t N = m.n_cells;
  r.off.resize(m.n_tiles);
  r.bytes.resize(m.n_tiles);
  r.ne_nh.resize(m.n_tiles);
  r.flags.assign(m.n_tiles, 0);
  std::vector<int32_t> halo;
  for (int64_t tile = 0; tile < m.n_tiles; ++tile) {
    const int64_t base = tile * kTile;
    const int64_t e0 = m.eoff[tile], e1 = m.eoff[tile + 1];
    const uint32_t ne = static_cast<uint32_t>(e1 - e0);
    if (ne > static_cast<uint32_t>(kMaxTileEdges)) return fail(BM_EINVAL, "tile records: too many tile edges");
    auto in_tile = [&](int64_t g) { return g >= base && g < base + kTile; };
    halo.clear();
    for (int64_t e = e0; e < e1; ++e) {
      if (!in_tile(m.eL[e])) halo.push_back(m.eL[e]);
      if (m.eR[e] >= 0 && !in_tile(m.eR[e])) halo.push_back(m.eR[e]);
    }
    std::sort(halo.begin(), halo.end());
    halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
    const uint32_t nh = static_cast<uint32_t>(halo.size());
    if (kTile + nh > static_cast<uint32_t>(kMaxLocal)) return fail(BM_EINVAL, "tile records: halo too large");
    auto local = [&](int64_t g) -> uint32_t {
      if (in_tile(g)) return static_cast<uint32_t>(g - base);
      return kTile + static_cast<uint32_t>(std::lower_bound(halo.begin(), halo.end(), g) - halo.begin());
    };
    const uint32_t ne4 = round4(ne), nh4 = round4(nh);
    const uint32_t bytes = RL::bytes(ne4, nh4);
    const size_t at = r.data.size();
    r.data.resize(at + bytes, 0);
    r.off[tile] = at;
    r.bytes[tile] = bytes;
    r.ne_nh[tile] = ne | (nh << 16);
    r.ne4_max = std::max(r.ne4_max, ne4);
    r.nh4_max = std::max(r.nh4_max, nh4);
    std::vector<uint32_t> lr(ne);
    for (uint32_t k = 0; k < ne; ++k) {
      const int64_t e = e0 + k;
      const int32_t gR = m.eR[e];
      int32_t R;
      if (gR >= 0) {
        R = static_cast<int32_t>(local(gR));
      } else {
        if (gR < kMinCode) return fail(BM_EINVAL, "tile records: too many listed boundary edges");
        R = gR;
        const int64_t j = kInflow - gR;  // listed edge (j >= 0) or a wall / transmissive code
        if (gR != kWall)  // walls carry no mass: a tile of walls only is an interior tile
          r.flags[tile] |= j < 0 ? 1
                                 : (j < m.n_inflow ? 3
                                                   : (j < m.n_inflow + m.n_hq ? 9
                                                                              : (j < m.n_inflow + m.n_hq + m.n_weir ? 17 : 33)));
      }
      lr[k] = local(m.eL[e]) | (static_cast<uint32_t>(R) << kLocBits);
      put<uint32_t>(r.data, at + RL::lr() + 4 * k, lr[k]);
      put<T>(r.data, at + RL::nx(ne4) + S * k, static_cast<T>(m.enx[e]));
      put<T>(r.data, at + RL::ny(ne4) + S * k, static_cast<T>(m.eny[e]));
      put<T>(r.data, at + RL::len(ne4) + S * k, static_cast<T>(m.elen[e]));
    }
    for (uint32_t h = 0; h < nh; ++h) put<int32_t>(r.data, at + RL::hidx(ne4) + 4 * h, halo[h]);
    for (int j = 0; j < kTile; ++j) {
      const int64_t i = base + j;
      put<T>(r.data, at + RL::ia() + S * j, static_cast<T>(m.inv_area[i]));
      if (i >= N) continue;
      uint32_t slot = 0;
      for (int k = 0; k < 3; ++k) {
        const uint32_t p = static_cast<uint32_t>((m.slots[i] >> (16 * k)) & 0xffffu);
        const uint32_t pos = p >> 1, side = p & 1u;
        if (pos >= ne) return fail(BM_EINVAL, "tile records: slot outside the tile's edge list");
        // the side must follow from the edge's left index
        const bool left = (lr[pos] & (kMaxLocal - 1)) == static_cast<uint32_t>(j);
        if (left != (side == 0)) return fail(BM_EINVAL, "tile records: inconsistent edge side");
        slot |= pos << (kLocBits * k);
      }
      put<uint32_t>(r.data, at + RL::slot() + 4 * j, slot);
    }
  }
  return BM_OK;
}
}  // namespace

bm_status build_tile_records(const HostMesh& m, int S, TileRecords* out) {
  try {
    if (S == 8) return build_records_t<double>(m, out);
    if (S == 4) return build_records_t<float>(m, out);
  } catch (const std::bad_alloc&) {
    return fail(BM_ENOMEM, "tile records: out of host memory");
  }
  return fail(BM_EINVAL, "tile records: element size must be 4 or 8");
}

}  // namespace bm
