"""Seeded synthetic detector frames (stand-ins for the paper's LCLS runs).

This package holds no step of the compression method: it only draws inputs.
Both the CUDA path (through its tests and the benchmark) and the CPU oracle
take their frames from here.
"""
from .frames import (GEOMETRIES, FrameRecipe, RECIPES, make_frame, make_batch,
                     make_batch_threaded)

__all__ = ["GEOMETRIES", "FrameRecipe", "RECIPES", "make_frame", "make_batch",
           "make_batch_threaded"]
