// Internal declarations of libnyxrt: constants of the exact traversal,
// device-side record layouts and kernel launchers. Not part of the ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/nyxrt.h"

#include "spectrum.h"

namespace nyx {

// Ray directions are HEALPix pixel centres quantised to 2^-kDirBits per
// component; the split radius R_0 = sqrt(3 / (pi N_min)) is quantised to
// 2^-kRadBits cells. With these, every traversal decision (next face, start
// cell, reaching the split sphere) is an exact integer comparison.
constexpr int kDirBits = 21;
constexpr int kRadBits = 24;
constexpr int kMaxLevel = 13;          // level cap: ray ids pack the pixel in 31 bits
constexpr double kSqrtPiOver3 = 1.0233267079464885;  // pixel width = r sqrt(Omega(l))

// One emitted source (after dedup / merge), 32 bytes.
struct SrcEntry {
    int32_t cx, cy, cz, pad;
    double ph;        // photons/s per unit ray budget: Ndot / 12
    double gd;        // rate scale per unit budget per cell of path: ph * sigma / dx^2 (FP64 march)
    float gf;         // the same rounded to float (FP32 march)
    float pad2;
};

// Device-side statistics and photon ledger, accumulated with atomics.
struct DevStats {
    unsigned long long rays[RT_MAX_LEVELS];
    unsigned long long splits[RT_MAX_LEVELS];
    unsigned long long escaped[RT_MAX_LEVELS];
    unsigned long long dropped_tau[RT_MAX_LEVELS];
    unsigned long long dropped_level[RT_MAX_LEVELS];
    unsigned long long segments[RT_MAX_LEVELS];
    unsigned long long secondary[RT_MAX_LEVELS];
    unsigned long long visit_hash;
    double absorbed, escaped_ph, dropped_ph;
    // -- fields below survive the per-trace reset (which clears up to `deposited`)
    double deposited;
    double emitted;
    double maxdiff;                  // chemistry: max |<x>_new - <x>_old| (as ordered bits)
    double xsum;                     // sum of x (automerge)
    unsigned int err;                // RT_ERR_* bits set by kernels
    unsigned int bad_input;          // count of invalid field / source values
};

enum : unsigned {
    kErrRayOverflow = 1u,            // next-level ray buffer too small
    kErrUnionFind = 2u,              // union-find retry cap reached
    kErrLevel = 4u,                  // a ray exceeded the direction table
    kErrGeometry = 8u,               // a geometry-table entry could not be encoded or ran out
};

// Ray records between levels (structure of arrays). A record is a parent
// that reached its split sphere; its four children are implicit
// (pixel 4p + q, budget P/4, same tau).
template <class R>
struct RayBuf {
    uint32_t* src = nullptr;
    uint32_t* pix = nullptr;
    R* P = nullptr;
    R* tau = nullptr;
    float* cP = nullptr;             // Kahan compensation terms (FP32 march only)
    float* ctau = nullptr;
    int64_t cap = 0;
};

template <class R>
struct MarchArgs {
    int level;
    int n;
    int64_t c0, c1;                  // child range [c0, c1) of this launch
    const int4* dirs;                // direction table of this level: {sdx, sdy, sdz, float_as_int(nrm)}
    const SrcEntry* src;
    RayBuf<R> in;                    // parents (unused at level 0)
    RayBuf<R> out;                   // next-level parents
    unsigned long long* out_count;
    const R* kap;                    // signed kappa: sign bit set = not eligible as Eq. 7-8 neighbour
    double* gamma;
    int64_t rq;
    int level_max;
    R tau_max;
    int overlap_mode;
    int hash;
    long long rs;                    // periodic boundaries: travel-distance cutoff (2^-24 cells); 0: none
    SpecTable<R> spec;               // RT_SPECTRUM_BLACKBODY pieces; spec.lin_a null: gray
    DevStats* st;
    // parents of this level counted on the device (written by the previous level's launch): the
    // launch then covers children [c0, min(c1, c0 + 4 * *in_count)); null: [c0, c1) as given
    const unsigned long long* in_count = nullptr;
};

// Geometry table of one level (FP32 march): 8-byte entries, entry s of pixel p at
// ent[(row0[p / 32] + s) * 32 + p % 32].
struct GeomLevel {
    const uint2* ent = nullptr;              // FP32 march: 8-byte entries
    const ulonglong2* ent64 = nullptr;       // FP64 march: 16-byte entries at the same row offsets
    const unsigned long long* row0 = nullptr;
};

// One solve of a batch, as the batch kernel sees it.
struct BatchSolve {
    const void* kap;         // float or double kappa of this solve
    double* gamma;
    DevStats* st;
    int n;
    int level_max;
    int overlap_mode;
    int hash;
    long long rq;
    double tau_max;
    uint32_t src_off;        // index of this solve's first source in the batch catalog
    uint32_t pad_;
    long long rs;            // periodic boundaries: travel-distance cutoff (2^-24 cells); 0: none
};

template <class R>
struct BatchArgs {
    const BatchSolve* solves;
    const SrcEntry* src;             // the launch's emitted sources; SrcEntry::pad = solve index
    long long nsrc;
    unsigned src_base;               // batch-catalog index of src[0]
    const int4* dirs;                // direction table from level 0
    int table_level;
    RayBuf<R> buf[RT_MAX_LEVELS + 1];  // parents of level l live in buf[l]
    long long slice;                 // children per slice (<= every buffer's capacity)
    int tile;                        // children per claimed tile (multiple of 32)
    unsigned long long* counts;      // per slice: next-level records written (zeroed)
    unsigned long long* tiles;       // per slice: tiles claimed (zeroed)
    int max_slices;
    int any_hash;                    // some solve asks for the visit hash
    int use_geo;                     // every solve shares rq and every level is tabled: geometry from the tables below
    GeomLevel geo[RT_MAX_LEVELS + 1];
    int single;                      // the launch holds one solve, given in `one`
    BatchSolve one;
    unsigned* err;
    int freq;                        // every solve of the launch takes the blackbody rate of `spec`
    SpecTable<R> spec;
};

// march.cu
int launch_march_f64(const MarchArgs<double>& a, int grid, int block, cudaStream_t s);
int launch_march_f32(const MarchArgs<float>& a, int grid, int block, cudaStream_t s);
cudaError_t launch_batch_f64(const BatchArgs<double>& a, int grid, int block, cudaStream_t s);
cudaError_t launch_batch_f32(const BatchArgs<float>& a, int grid, int block, cudaStream_t s);
int batch_blocks_per_sm(int precision, int block, bool table, bool single, bool freq);
// The march of one level with its geometry from a table (FP32: g.ent; FP64: g.ent64).
int launch_march_table_f32(const MarchArgs<float>& a, const GeomLevel& g, int grid, int block, cudaStream_t s);
int launch_march_table_f64(const MarchArgs<double>& a, const GeomLevel& g, int grid, int block, cudaStream_t s);
// Geometry-table generation for level l of directions dirs (npix pixels), for grids up to
// n_cover: rows[b] = rows of 32-pixel block b; then the entries at row offsets row0.
// rs: travel-distance cutoff of periodic boundaries (0: none).
void launch_geom_count(long long rq, int l, const int4* dirs, long long npix, int n_cover, long long rs,
                       unsigned* rows, cudaStream_t s);
void launch_geom_fill(long long rq, int l, const int4* dirs, long long npix, int n_cover, long long rs,
                      const unsigned long long* row0, uint2* ent, unsigned* err, cudaStream_t s);
// The FP64 entries of the same level at the same row offsets (total rows: rows_total).
void launch_geom_fill64(long long rq, int l, const int4* dirs, long long npix, int n_cover, long long rs,
                        const unsigned long long* row0, unsigned long long rows_total, ulonglong2* ent,
                        unsigned* err, cudaStream_t s);

// fields.cu
int launch_validate_fields(const double* nh, const double* x, int64_t ncell, DevStats* st, cudaStream_t s);
int launch_prepare_kappa_f64(const double* nh, const double* x, int64_t ncell, double sdx, double n_th,
                              double* kap, cudaStream_t s);
int launch_prepare_kappa_f32(const double* nh, const double* x, int64_t ncell, double sdx, double n_th,
                              float* kap, cudaStream_t s);
int launch_finalize(const double* gamma, const double* nh, const double* x, int64_t ncell, double e_heat,
                     double vol, double* heat, DevStats* st, cudaStream_t s);
int launch_chem_update(const double* nh, const double* x0, double* xavg, double* xend, const double* gamma,
                        int64_t ncell, double dt, double alpha_B, double C_H, double clump, DevStats* st,
                        cudaStream_t s);
int launch_sum_x(const double* x, int64_t ncell, DevStats* st, cudaStream_t s);
int launch_mean_nh(const double* nh, int64_t ncell, double* out, cudaStream_t s);

// Small device-to-host readbacks (statistics, counters), written by one kernel straight into mapped
// pinned host memory: unlike copies they do not queue on the copy engines behind large transfers
// that other streams have in flight. Up to four regions, each a whole number of 4-byte words; dst
// holds device addresses of pinned host memory.
struct ReadbackList {
    const unsigned* src[4] = {};
    unsigned* dst[4] = {};
    int words[4] = {};
    int n = 0;
    void add(const void* from, void* to, size_t bytes)
    {
        src[n] = static_cast<const unsigned*>(from);
        dst[n] = static_cast<unsigned*>(to);
        words[n] = (int)(bytes / 4);
        ++n;
    }
};
int launch_readback(const ReadbackList& r, cudaStream_t s);

// sources.cu
struct SourceWork {
    int32_t* cells_raw = nullptr;   // cap x 3, appended sources
    double* ndot_raw = nullptr;     // cap
    uint64_t* keys = nullptr;       // scratch, cap
    uint64_t* keys_b = nullptr;     // sort scratch, cap
    uint64_t* keys_c = nullptr;     // sort scratch, cap
    int32_t* order = nullptr;       // scratch, cap
    int32_t* order_b = nullptr;     // sort scratch, cap
    int32_t* flag = nullptr;        // scratch, cap
    int32_t* head_pos = nullptr;    // scratch, cap
    int32_t* cells_a = nullptr;     // cap x 3: deduplicated (then merged) sorted catalog
    double* ndot_a = nullptr;       // cap
    int32_t* cells_b = nullptr;     // cap x 3: merge scratch
    double* ndot_b = nullptr;       // cap
    int32_t* label = nullptr;       // cap: union-find root of each source
    int* parent = nullptr;          // cap: union-find forest
    double* radius = nullptr;       // cap: Alg. 3 bubble radii
    int32_t* count = nullptr;       // device scalars [4]
    int64_t cap = 0;
};
int launch_validate_sources(const int32_t* cells, const double* ndot, int64_t nsrc, int n, DevStats* st,
                             cudaStream_t s);
// Dedup + lexicographic sort (cells of an n^3 grid); writes cells_a/ndot_a and count[0] = number
// of unique cells.
int launch_dedup_sort(SourceWork& w, int64_t nsrc, int n, cudaStream_t s);
// Alg. 3 on cells_a/ndot_a[0..m): radii, union-find, merged catalog into cells_a/ndot_a, count[0] = size.
int launch_merge(SourceWork& w, int64_t m, int n, int periodic, const double* x, const int4* samp_dirs,
                 int samp_count, double x_th, double f_req, int n_min, double dr, double rmax, double f_ov,
                 double eps, DevStats* st, cudaStream_t s);
// Emitted catalog entries from cells_a/ndot_a[0..*count) with *count read on the device (<= max_m).
int launch_build_emit_dev(const SourceWork& w, int64_t max_m, double s_over_dx2, SrcEntry* out, DevStats* st,
                          cudaStream_t s);
// Emitted catalog entries from cells_a/ndot_a[0..m).
int launch_build_emit(const SourceWork& w, int64_t m, double s_over_dx2, SrcEntry* out, DevStats* st,
                      cudaStream_t s);

// directions.cpp: quantised HEALPix nested pixel centres, levels 0..max_level
// concatenated (offset of level l = 12 (4^l - 1) / 3). Host memory.
void healpix_direction_table(int max_level, int4* out);
int64_t healpix_level_offset(int level);

}  // namespace nyx
