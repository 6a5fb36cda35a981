// Forward projector P: launch geometry and shared-memory sizing common to the host
// dispatcher (project.cu) and the kernel's instantiations (project_kernel.cuh).
#pragma once
#include <cstddef>

#include "cbct_internal.cuh"

namespace cbct {

constexpr int PROJ_THREADS = 192; // threads per block; each thread walks two imager rows
#ifndef CBCT_PROJ_MIN_BLOCKS
// resident blocks per SM the register budget is sized for (at most 64 registers a thread;
// no spills): a fifth block hides more of the phases' shared-memory latency than the
// registers it costs (measured: 15-22% on the paper's coarser multigrid levels)
#define CBCT_PROJ_MIN_BLOCKS 5
#endif
constexpr float P_INF = 3.0e38f;

// threads of a block (a multiple of 32, every lane present for warp votes) and the imager
// rows one block covers (two per thread)
static inline int proj_threads(const GeomDev &G)
{
    const int rows = G.nv < 2 * PROJ_THREADS ? G.nv : 2 * PROJ_THREADS;
    const int t = (((rows + 1) / 2 + 31) / 32) * 32;
    return t < PROJ_THREADS ? t : PROJ_THREADS;
}

// segments of a trace (at most nx + ny + 1), padded to whole groups
static inline int seg_capacity(const GeomDev &G, int sg)
{
    return ((G.nx + G.ny + 2 + sg - 1) / sg) * sg;
}

// Shared memory of one block: the two crossing lists, then (16-byte aligned) per segment
// its end tau, its column offset and the packed record used by the walk.
static inline int seg_offset(const GeomDev &G) { return ((G.nx + G.ny + 2 + 3) / 4) * 4; }

// z-lines of one group of columns, staged in shared memory one line per column. A column
// starts at float offset col of the z-contiguous volume; its line is copied in 16-byte
// pieces from col rounded down to a multiple of 4 up to col + nz rounded up, i.e. at most
// nz + 6 floats, and the column's first voxel sits at (col & 3) in its line. The copy may
// read up to 3 floats past the last voxel of the volume: every volume buffer the
// projector reads has at least 16 bytes of slack after it (PROJECT_VOLUME_SLACK).
static inline int line_pitch(int nz) { return ((nz + 6 + 3) / 4) * 4; }

// shared memory: per segment (end tau, column offset, (line offset, length)); then the
// staged z-lines of one group, whose space first holds phase 1's crossing lists; then the
// group's per-slab prefix table and two rows of running per-slab totals
static inline size_t line_region(const GeomDev &G, int sg)
{
    const size_t lines = (size_t)sg * line_pitch(G.nz), lists = (size_t)seg_offset(G);
    return lines > lists ? lines : lists;
}

static inline size_t project_smem(const GeomDev &G, int sg)
{
    return (sizeof(float) + sizeof(int) + sizeof(float2)) * (size_t)seg_capacity(G, sg) +
           sizeof(float) * (line_region(G, sg) + (size_t)G.nz * (sg + 1) + 2 * (size_t)G.nz);
}

// The trace table (k_trace_table): a record of 16 + 8 trace_cap bytes per (view, imager
// column), trace_cap = nx + ny + 2 rounded up to 4.
static inline int trace_cap(const GeomDev &G) { return ((G.nx + G.ny + 2 + 3) / 4) * 4; }
static inline size_t trace_smem(const GeomDev &G)
{
    return sizeof(float) * (2 * (size_t)trace_cap(G) + 4 * (PROJ_THREADS / 32) + (size_t)G.nx + G.ny + 2);
}

// Column segments per group (one staged set of z-lines and one prefix table); the
// dispatcher (project.cu) picks one per launch from an estimate of its per-group cost and
// of the blocks it keeps resident.
constexpr int PROJECT_GROUP_SIZES[] = {16, 24, 32, 40, 48, 56, 64, 80, 96};
constexpr int PROJECT_N_GROUP_SIZES = (int)(sizeof(PROJECT_GROUP_SIZES) / sizeof(int));

// The instantiation k_project<MODE, TP, SG> for a mode and storage type (host address
// for cudaLaunchKernel and the attribute and occupancy queries), or nullptr where it is
// not compiled: PM_COUNT walks the trace without groups and exists for SG = 16 only.
// Defined for each SG of PROJECT_GROUP_SIZES in the project_groups_*.cu units.
template <int SG> const void *project_kernel(int mode, int storage);

} // namespace cbct
