"""Seeded synthetic YUV 4:2:0 frames (inputs only; no analyzer arithmetic here)."""

from .frames import *  # noqa: F401,F403
