// Host-side scene preparation: mesh validation, boundary surface, lumped mass,
// rest-shape inverses and the MAS subdomain hierarchy (supplement Sec. 1.2).
#pragma once
#include <string>
#include <vector>

#include "ipc.h"

namespace ipcb {

constexpr int kSub = 32;      // nodes per MAS subdomain -> 96x96 blocks
constexpr int kBlk = 3 * kSub;
constexpr int kMaxLevels = 6;

struct HostMesh {
    int nv = 0, nt = 0;
    std::vector<double> x_rest, x0, v0;
    std::vector<int> tets;
    std::vector<double> mass, vol, mu, lam, dminv;  // dminv: 9 per tet, row-major
    // boundary surface in lexicographic order of sorted vertex ids
    std::vector<int> sv, sf, se;
    std::vector<int> vert_adj_ptr, vert_adj;
    // connected components of the tet mesh, numbered by their lowest vertex id
    int nbody = 0;
    std::vector<int> body;
    // hierarchy: level l has nnodes[l] nodes in ngroups[l] groups of <= 32
    int nlev = 0;
    std::vector<int> nnodes, ngroups;
    std::vector<std::vector<int>> group_of, slot_of, members, node_of_vert;
    double bbox_diag = 0.0;
    double mean_surface_edge = 0.0;
    double max_surface_edge = 0.0;
    double gravity[3] = {0, 0, 0};
    int has_ground = 0;
    double gn[3] = {0, 1, 0}, goff = 0.0;
};

// Returns 0 on success, else an ipc_status with *err filled.
int build_host_mesh(const ipc_scene_desc* d, int levels_max, HostMesh* m, std::string* err);

}  // namespace ipcb
