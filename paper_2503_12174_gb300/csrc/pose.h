// pose.h -- launchers of the camera-pose gradient (pose.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace dpcs {

// One mesh edge for the silhouette term, in increasing (lower vertex, higher
// vertex) order of the original mesh: x = leaf position of the triangle whose
// third vertex has the lower index (-1: the edge has more than two triangles
// and is skipped), y = its corners of the lower vertex, the higher vertex and
// the third vertex (2 bits each, in that order), z = leaf position of the
// other triangle (-1: a boundary edge), w = that triangle's third corner.
using PoseEdge = int4;

// Arguments the pose kernels take beside RenderArgs.
struct PoseArgs {
    float Kc[9];            // camera intrinsics (row-major)
    int32_t edge_spp;       // samples per pixel edge (0 = no pixel-edge term)
    int32_t sil_spp;        // samples per silhouette edge (0 = no silhouette term)
    const PoseEdge *edges;  // mesh edges (null when sil_spp == 0)
    int64_t nedges;
    double *partial;        // 3 x pose_grid(device) x 6 per-block sums
    const float4 *mat;      // the principled material's packed maps (metallic, normal map), or null: plain
};

// blocks of each pose kernel on this device (its partial sums are 6 per block)
int pose_grid(int device);
// interior, pixel-edge and silhouette terms; wrench (18 FP64) += their sums.
// Returns the kernels enqueued or a negative dpcs_status.
int launch_pose(const RenderArgs &a, const PoseArgs &p, int device, double *wrench, cudaStream_t st);

}  // namespace dpcs
