"""Seeded synthetic inputs for radiance-texture shading.

This package is shared by the tests, the oracle checks and the benchmark.  It
holds only scene generation (analytic ray casting of a G-buffer: UV,
tangent-space view direction, object id) and seeded draws of field
parameters.  It holds none of the method's arithmetic: no equisolid
projection, no disc-to-square mapping, no filtering.  All draws use numpy's
PCG64 generator with the seed given by the caller, and geometry is computed in
FP64 then rounded to FP32, the G-buffer precision.
"""
from .scenes import (GBuffer, quad_scene, quad_views, sphere_plane_poses, sphere_plane_scene,  # noqa: F401
                     voronoi_planes_scene)
from .fields import (PATTERN_A, PATTERN_B, PATTERN_K, PATTERN_M, bucket_lobe_params,  # noqa: F401
                     eval_field_lobes, field_lobes, pattern_values)
from .bake import ao_directions, bake_scene  # noqa: F401
