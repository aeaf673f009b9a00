"""Seeded input generators (no hull arithmetic); see ``synth.workloads``."""
from .workloads import *  # noqa: F401,F403
