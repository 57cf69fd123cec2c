// sgtp_batch.hpp -- the race table of an sgtp_batch, shared by the planning
// and the closed-loop simulation translation units.
#pragma once

#include <vector>

#include "sgtp_host.hpp"

namespace sgtp {

// One race of a batch on the device: its sizes and the offsets of its
// slices in the batch arrays.
struct RaceDev {
    int track_id, n_v, T, ego;
    unsigned race_tag;
    int n_tail;
    int agent_off;   // first vehicle of the race in the batch arrays
    int u_off;       // float offset into U_io (n_v * T * 2 per race)
    int xi_off;      // float offset into xi_out (n_v * (T+1) * 4)
    int ks_off;      // offset into k_star_out ((L+1) * n_v + 1)
    int pos_off;     // float2 offset into each prediction buffer (n_v * (T+1))
    int pad0;
    // work before this race in a round per sample tile of a vehicle (each
    // tile of a race weighs its horizon T; a launch multiplies by its tiles
    // per vehicle): Jacobi rounds (every vehicle) and the extra round (egos)
    long long wcum_all, wcum_ego;
};

}  // namespace sgtp

struct sgtp_batch {
    const sgtp_track *trk = nullptr;
    int n_races = 0, K = 0, L = 0;
    std::vector<sgtp::RaceDev> races;
    sgtp::RaceDev *races_dev = nullptr;
    long long agents = 0, u_elems = 0, xi_elems = 0, ks = 0, n_pos = 0;
    int maxT = 0, max_nv = 0;
    int minT = 0;   // shortest horizon of the batch's races
    long long w_all = 0, w_ego = 0;   // total work of a Jacobi round / the extra round (see RaceDev)
};

