"""GB300-native grasp-search hot path of Fast-Grasp'D (arXiv 2306.08132).

The compute lives in libfastgraspd.so (hand-written CUDA for sm_103a behind the
C ABI of include/fastgraspd.h); this package is its thin Python binding.
"""

from . import _lib
from .autograd import GraspLoss, grasp_loss
from .api import (Hand, Sdf, Scene, make_params, fk, sdf_query, contact_wrench, loss_and_grad,
                  optimize_step, optimize_step_plain, plain_workspace_size, fused_configs, fused_config_select,
                  fused_config_current, autotune, Queue,
                  optimize_step_plain_noalloc, contact_measure, grasp_epsilon, fp32_peak_launch, optimize_step_host, test_fail_allocation)

__all__ = ["GraspLoss", "grasp_loss", "Hand", "Sdf", "Scene", "make_params", "fk", "sdf_query", "contact_wrench", "loss_and_grad",
           "optimize_step", "optimize_step_plain", "plain_workspace_size", "fused_configs",
           "fused_config_select", "fused_config_current", "autotune", "Queue",
           "optimize_step_plain_noalloc", "contact_measure", "grasp_epsilon", "fp32_peak_launch", "optimize_step_host", "test_fail_allocation"]
