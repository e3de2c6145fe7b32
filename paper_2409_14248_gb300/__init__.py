"""HRKAN physics-informed training on GB300 (sm_103a)."""
