// Observables at sample times (Sec. 2.1): occupation spectra n_m(k), transverse spin
// structure factor S_perp(k), radially binned, plus norm and energy diagnostics, all
// accumulated in FP64 with a fixed reduction order.
#pragma once

#include <vector>

#include "gpe.h"
#include "internal.h"

namespace gpe {

// Radial bins of one shape group: its spectra sit in each accumulator slot at
// 4 * offset doubles, laid out [field][bin] over its nbins bins.
struct GroupBins {
    int nbins = 0;                   // 0: no spectra for the group (unequal side lengths)
    int64_t offset = 0;              // bins of the groups before it
    int32_t* d_off = nullptr;        // CSR offsets over bins (nbins + 1)
    int32_t* d_modes = nullptr;      // mode indices sorted by bin, then by index
};

struct ObsWork {
    int nbins = 0;                   // radial bins of all groups (0: spectra unavailable for this batch)
    std::vector<int64_t> counts;     // modes per bin, the groups' bins one after the other
    std::vector<GroupBins> gbins;    // per shape group
    void* d_W = nullptr;             // workspace: chunk x 4 fields x sites complex
    void** d_Wptrs = nullptr;        // per chunk slot: its 4-field block
    double* d_part = nullptr;        // chunk x nblk x 7 real-space partial sums
    double* d_ekin = nullptr;        // chunk x 3 x nblk kinetic partial sums
    int64_t chunk = 0;               // trajectories per workspace chunk
    int64_t nblk = 0;                // site blocks per trajectory (largest group)
    int64_t ntraj_total = 0;
    bool f64 = false;
    bool ready = false;              // workspace allocated
};

gpe_status obs_init(ObsWork& w, const std::vector<Group>& groups, bool f64, int device);
void obs_free(ObsWork& w);
gpe_status obs_accumulate(ObsWork& w, const std::vector<Group>& groups, bool f64, double c0, double c1,
                          double q, double* acc, uint32_t flags, int slot, int* d_status, cudaStream_t s);
const char* obs_last_error();
// Kernels one obs_accumulate call launches (for the launch counter).
int64_t obs_launches(const ObsWork& w, const std::vector<Group>& groups, uint32_t flags);

}  // namespace gpe
