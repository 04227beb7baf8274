"""GB300-native log-polar Radon transform and back-projection (arXiv 1506.00014).

The transforms run in hand-written CUDA kernels for sm_103a inside ``libradon.so``
(C ABI in ``include/radon.h``); ``binding`` marshals arguments to it.
"""

from .binding import (  # noqa: F401
    RADON_FILTER_COSINE,
    RADON_FILTER_RAMP,
    RADON_FILTER_SHEPP_LOGAN,
    RadonError,
    RadonPlan,
    load,
    radon_backproject,
    radon_backproject_batch,
    radon_backproject_host,
    radon_backproject_multi,
    radon_fbp,
    radon_forward,
    radon_forward_batch,
    radon_forward_host,
    radon_forward_multi,
    radon_forward_static_scratch,
    radon_geometry,
    radon_kernel_quadrant,
    radon_plan_create,
    radon_plan_destroy,
    radon_plan_get_info,
    radon_plan_reserve_batch,
    radon_plan_set_column_group,
    radon_plan_kernel_launches,
    radon_profile_enable,
    radon_profile_read,
    radon_status_string,
    radon_transpose,
    radon_transpose_batch,
)
