// Host-side scene preparation (see host_mesh.h).
//
// Readings shared with the method description: lumped mass rho V / 4 per tet
// vertex; Lame parameters mu = E / (2 (1 + nu)), lambda = E nu / ((1 + nu)(1 -
// 2 nu)); the surface is the set of tet faces used once; subdomains are runs of
// 32 nodes of a greedy BFS over mesh adjacency that starts at the lowest
// unvisited node and visits neighbours in ascending order; level l+1 nodes
// are level-l subdomains, adjacent when a mesh edge joins them; a level with
// at most 32 nodes is one subdomain and the last (at most levels_max levels).
#include "host_mesh.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <deque>

namespace ipcb {

namespace {

// Ascending neighbour lists from a list of directed pairs (u, w).
void pairs_to_csr(int n, std::vector<std::pair<int, int>>& pr, std::vector<int>& ptr, std::vector<int>& nb) {
    std::sort(pr.begin(), pr.end());
    pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
    ptr.assign(n + 1, 0);
    nb.resize(pr.size());
    for (size_t i = 0; i < pr.size(); ++i) {
        ptr[pr[i].first + 1]++;
        nb[i] = pr[i].second;
    }
    for (int i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
}

std::vector<int> bfs_order(int n, const std::vector<int>& ptr, const std::vector<int>& nb) {
    std::vector<int> order;
    order.reserve(n);
    std::vector<char> seen(n, 0);
    std::deque<int> q;
    for (int s = 0; s < n; ++s) {
        if (seen[s]) continue;
        seen[s] = 1;
        q.push_back(s);
        while (!q.empty()) {
            int u = q.front();
            q.pop_front();
            order.push_back(u);
            for (int k = ptr[u]; k < ptr[u + 1]; ++k)
                if (!seen[nb[k]]) {
                    seen[nb[k]] = 1;
                    q.push_back(nb[k]);
                }
        }
    }
    return order;
}

}  // namespace

int build_host_mesh(const ipc_scene_desc* d, int levels_max, HostMesh* m, std::string* err) {
    if (!d || d->n_verts <= 0 || d->n_tets <= 0 || !d->x_rest || !d->tets || !d->E || !d->nu || !d->rho) {
        *err = "scene: empty mesh or missing arrays";
        return IPC_ERR_INVALID;
    }
    const int nv = d->n_verts, nt = d->n_tets;
    m->nv = nv;
    m->nt = nt;
    m->x_rest.assign(d->x_rest, d->x_rest + 3 * (size_t)nv);
    m->x0.assign(d->x0 ? d->x0 : d->x_rest, (d->x0 ? d->x0 : d->x_rest) + 3 * (size_t)nv);
    if (d->v0)
        m->v0.assign(d->v0, d->v0 + 3 * (size_t)nv);
    else
        m->v0.assign(3 * (size_t)nv, 0.0);
    m->tets.assign(d->tets, d->tets + 4 * (size_t)nt);
    for (int i = 0; i < 4 * nt; ++i)
        if (m->tets[i] < 0 || m->tets[i] >= nv) {
            *err = "scene: tet vertex id out of range";
            return IPC_ERR_INVALID;
        }
    for (size_t i = 0; i < m->x0.size(); ++i)
        if (!std::isfinite(m->x0[i]) || !std::isfinite(m->x_rest[i]) || !std::isfinite(m->v0[i])) {
            *err = "scene: non-finite coordinate";
            return IPC_ERR_INVALID;
        }

    // rest shapes, volumes, materials, lumped mass
    m->mass.assign(nv, 0.0);
    m->vol.resize(nt);
    m->mu.resize(nt);
    m->lam.resize(nt);
    m->dminv.resize(9 * (size_t)nt);
    for (int t = 0; t < nt; ++t) {
        const int* q = &m->tets[4 * t];
        double A[3][3];  // columns X_j - X_0
        for (int j = 0; j < 3; ++j)
            for (int r = 0; r < 3; ++r) A[r][j] = m->x_rest[3 * q[j + 1] + r] - m->x_rest[3 * q[0] + r];
        double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
        double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
        double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
        double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
        if (!(det > 0.0)) {
            *err = "scene: tet " + std::to_string(t) + " has non-positive rest volume";
            return IPC_ERR_INVALID;
        }
        double inv[3][3];
        inv[0][0] = c00 / det;
        inv[1][0] = c01 / det;
        inv[2][0] = c02 / det;
        inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
        inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
        inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
        inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
        inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
        inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) m->dminv[9 * (size_t)t + 3 * r + c] = inv[r][c];
        double V = det / 6.0;
        m->vol[t] = V;
        double E = d->E[t], nu = d->nu[t];
        if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5) || !(d->rho[t] > 0.0)) {
            *err = "scene: invalid material on tet " + std::to_string(t);
            return IPC_ERR_INVALID;
        }
        m->mu[t] = E / (2.0 * (1.0 + nu));
        m->lam[t] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        for (int j = 0; j < 4; ++j) m->mass[q[j]] += 0.25 * d->rho[t] * V;
    }
    for (int v = 0; v < nv; ++v)
        if (!(m->mass[v] > 0.0)) {
            *err = "scene: vertex " + std::to_string(v) + " belongs to no tet";
            return IPC_ERR_INVALID;
        }

    // boundary faces: sorted-id key + oriented triple; kept if used once
    struct Face {
        std::array<int, 3> key, tri;
    };
    static const int kFace[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};
    std::vector<Face> faces(4 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int f = 0; f < 4; ++f) {
            Face& F = faces[4 * (size_t)t + f];
            for (int j = 0; j < 3; ++j) F.tri[j] = m->tets[4 * t + kFace[f][j]];
            F.key = F.tri;
            std::sort(F.key.begin(), F.key.end());
        }
    std::sort(faces.begin(), faces.end(), [](const Face& a, const Face& b) { return a.key < b.key; });
    m->sf.clear();
    for (size_t i = 0; i < faces.size();) {
        size_t j = i + 1;
        while (j < faces.size() && faces[j].key == faces[i].key) ++j;
        if (j - i == 1) m->sf.insert(m->sf.end(), faces[i].tri.begin(), faces[i].tri.end());
        i = j;
    }
    const int nsf = (int)(m->sf.size() / 3);
    std::vector<std::pair<int, int>> edges;
    edges.reserve(3 * (size_t)nsf);
    std::vector<char> on_surf(nv, 0);
    for (int f = 0; f < nsf; ++f)
        for (int j = 0; j < 3; ++j) {
            int a = m->sf[3 * f + j], b = m->sf[3 * f + (j + 1) % 3];
            edges.emplace_back(std::min(a, b), std::max(a, b));
            on_surf[a] = 1;
        }
    std::sort(edges.begin(), edges.end());
    edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    m->se.clear();
    double elen = 0.0, emax = 0.0;
    for (auto& e : edges) {
        m->se.push_back(e.first);
        m->se.push_back(e.second);
        double s = 0.0;
        for (int r = 0; r < 3; ++r) {
            double dd = m->x_rest[3 * e.first + r] - m->x_rest[3 * e.second + r];
            s += dd * dd;
        }
        elen += std::sqrt(s);
        emax = std::max(emax, std::sqrt(s));
    }
    m->mean_surface_edge = edges.empty() ? 0.0 : elen / edges.size();
    m->max_surface_edge = emax;
    m->sv.clear();
    for (int v = 0; v < nv; ++v)
        if (on_surf[v]) m->sv.push_back(v);

    // vertex adjacency from tet edges
    std::vector<std::pair<int, int>> pr;
    pr.reserve(12 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                if (a != b) pr.emplace_back(m->tets[4 * t + a], m->tets[4 * t + b]);
    pairs_to_csr(nv, pr, m->vert_adj_ptr, m->vert_adj);

    // bodies: components over tet edges, numbered in order of lowest vertex
    m->body.assign(nv, -1);
    m->nbody = 0;
    {
        std::vector<int> stack;
        for (int v0 = 0; v0 < nv; ++v0) {
            if (m->body[v0] >= 0) continue;
            m->body[v0] = m->nbody;
            stack.push_back(v0);
            while (!stack.empty()) {
                int u = stack.back();
                stack.pop_back();
                for (int k = m->vert_adj_ptr[u]; k < m->vert_adj_ptr[u + 1]; ++k) {
                    int w = m->vert_adj[k];
                    if (m->body[w] < 0) {
                        m->body[w] = m->nbody;
                        stack.push_back(w);
                    }
                }
            }
            ++m->nbody;
        }
    }

    // hierarchy
    std::vector<int> ptr = m->vert_adj_ptr, nb = m->vert_adj;
    int n = nv;
    m->nlev = 0;
    m->nnodes.clear();
    m->ngroups.clear();
    m->group_of.clear();
    m->slot_of.clear();
    m->members.clear();
    m->node_of_vert.clear();
    for (int l = 0; l < levels_max && l < kMaxLevels; ++l) {
        bool last = (n <= kSub) || (l + 1 == levels_max) || (l + 1 == kMaxLevels);
        std::vector<int> order;
        if (n <= kSub) {
            order.resize(n);
            for (int i = 0; i < n; ++i) order[i] = i;
        } else {
            order = bfs_order(n, ptr, nb);
        }
        int ng = (n + kSub - 1) / kSub;
        std::vector<int> grp(n), slot(n), mem((size_t)ng * kSub, -1);
        for (int i = 0; i < n; ++i) {
            grp[order[i]] = i / kSub;
            slot[order[i]] = i % kSub;
            mem[i] = order[i];
        }
        std::vector<int> nov(nv);
        if (l == 0)
            for (int v = 0; v < nv; ++v) nov[v] = v;
        else
            for (int v = 0; v < nv; ++v) nov[v] = m->group_of[l - 1][m->node_of_vert[l - 1][v]];
        m->nnodes.push_back(n);
        m->ngroups.push_back(ng);
        m->group_of.push_back(std::move(grp));
        m->slot_of.push_back(std::move(slot));
        m->members.push_back(std::move(mem));
        m->node_of_vert.push_back(std::move(nov));
        m->nlev = l + 1;
        if (last) break;
        std::vector<std::pair<int, int>> cp;
        const std::vector<int>& G = m->group_of[l];
        for (int u = 0; u < n; ++u)
            for (int k = ptr[u]; k < ptr[u + 1]; ++k)
                if (G[u] != G[nb[k]]) cp.emplace_back(G[u], G[nb[k]]);
        pairs_to_csr(ng, cp, ptr, nb);
        n = ng;
    }

    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int v = 0; v < nv; ++v)
        for (int r = 0; r < 3; ++r) {
            lo[r] = std::min(lo[r], m->x_rest[3 * v + r]);
            hi[r] = std::max(hi[r], m->x_rest[3 * v + r]);
        }
    m->bbox_diag = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                             (hi[2] - lo[2]) * (hi[2] - lo[2]));
    for (int r = 0; r < 3; ++r) m->gravity[r] = d->gravity[r];
    m->has_ground = d->has_ground;
    if (m->has_ground) {
        double l = std::sqrt(d->ground_normal[0] * d->ground_normal[0] + d->ground_normal[1] * d->ground_normal[1] +
                             d->ground_normal[2] * d->ground_normal[2]);
        if (!(l > 0.0)) {
            *err = "scene: zero ground normal";
            return IPC_ERR_INVALID;
        }
        for (int r = 0; r < 3; ++r) m->gn[r] = d->ground_normal[r] / l;
        m->goff = d->ground_offset;
    }
    return IPC_OK;
}

}  // namespace ipcb
