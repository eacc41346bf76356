"""GB300-native fast multipole Legendre<->Chebyshev transform (arXiv:2411.00033).

Importing the package loads liblegcheb.so; build it first with
``paper_2411_00033_gb300.build.build()`` (or ``__graft_entry__.build()``).
"""
from . import binding  # noqa: F401
from .binding import (  # noqa: F401
    LC_L2C, LC_C2L, LC_F64, LC_F64_SPLIT, LC_F32, LC_F64_DF, LegChebError,
    lc_plan_workspace_size, lc_plan_create, lc_plan_workspace_size_ragged, lc_plan_create_ragged,
    lc_execute, lc_adjoint, lc_destroy, lc_status_string, lc_plan_info, lc_plan_table, lc_plan_launches,
)
from .api import Plan, get_plan, autotune_tile  # noqa: F401
from .autograd import leg2cheb, cheb2leg  # noqa: F401

binding.load()
