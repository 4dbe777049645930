// sphst_engine.cuh -- host side of one engine: the device arrays of a set of
// cases, the captured advection-step graph and its launch.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sphst.h"
#include "sphst_internal.cuh"

namespace sphst {

void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

struct Engine;

struct PhaseRec {
    sphst_phase_props props;
    int64_t first = 0, count = 0;
    int32_t fluid_index = -1;     // 0/1 for fluids, -1 for walls
};

// host record of one case
struct CaseRec {
    sphst_case_params P{};
    std::vector<PhaseRec> phases;
    std::vector<double> pos, vel, rho;     // staged input (3, 3, 1 per particle)
    std::vector<uint8_t> kind;             // 0/1 fluid, 2 wall
    int64_t n = 0, n_fluid = 0;
    int32_t n_fluid_phases = 0;
    double rho0[2] = {1.0, 1.0}, eta[2] = {1.0, 1.0};
    bool gridded = false;
    double origin[3] = {0, 0, 0}, cs = 0;
    int32_t ncell[3] = {1, 1, 1};
    int32_t bits = 0;
    int64_t table_size = 0;
    Engine *engine = nullptr;              // where the case lives (null: staged only)
    int32_t slot = -1;                     // index in the engine
    struct sphst_batch_s *batch = nullptr;
    cudaStream_t user_stream = nullptr;   // caller's stream, or null
    sphst_step_info info{};
};

// Fills the grid fields of a case from its staged positions (first step).
int make_grid(CaseRec *c);
// Device description of a case (both precisions).
CaseDesc make_desc(const CaseRec *c);
int map_status(int32_t dev_status);

struct Engine {
    int precision = 32;
    int refs = 0;
    std::vector<CaseRec *> members;
    virtual ~Engine() {}
    // allocate and fill from members (fresh ones from staged data, resident
    // ones by device copy from their current engine)
    virtual int setup(const std::vector<CaseRec *> &cases, int block, cudaStream_t user_stream) = 0;
    virtual int step(int64_t n_adv) = 0;
    virtual int profile_step(double *kernel_ms, int64_t *launches) = 0;
    virtual int sync_state() = 0;                       // copy CaseState -> members' info
    virtual int read_field(int slot, int field, double *host) = 0;
    virtual int debug_keys(int slot, uint64_t *keys, int64_t *ids) = 0;
    virtual int debug_counts(int slot, int32_t *counts) = 0;
    // FP64 reductions of one case (DIAG_Q doubles, layout of k_diag_final)
    virtual int diagnose(int slot, const double *center, double r_in, double r_out, double *q) = 0;
    // device copies used when a case moves to another engine
    virtual void *dev_array(int which) = 0;
    virtual CaseState *dev_state() = 0;
    virtual int64_t begin_of(int slot) = 0;
};

Engine *new_engine_f32();
Engine *new_engine_f64();
int64_t footprint(const sphst_case_params *P, int64_t n);

}  // namespace sphst
